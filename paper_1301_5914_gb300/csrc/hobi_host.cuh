// hobi_host.cuh -- host-side pieces shared by the C ABI translation units (hobi_capi.cu: the
// single-molecule handle; hobi_batch.cu: the batched handle): error reporting, the handle
// structure with its device tables and its matvec / GMRES pipelines, and the handle set-up the
// batch reuses for its molecules.
#pragma once

#include <math.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <new>
#include <stdio.h>
#include <stdlib.h>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hobi.h"
#include "hobi_internal.cuh"

namespace hobi {
namespace host {

// NVTX range around a public call (no-op unless a profiler is attached), so nsys / ncu timelines
// show setup, matvec, solve and energy phases by name.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// Message of the last failing call on this thread (hobi_last_error); defined in hobi_capi.cu.
extern thread_local std::string g_err;

inline int fail(int code, const std::string& msg) {
  try {
    g_err = msg;
  } catch (...) {  // out of host memory: keep the status, lose the message
  }
  return code;
}

// Runs a body that allocates host memory and turns a C++ exception (a failed host allocation,
// most likely) into a status, so that nothing throws across the C ABI.
template <class F>
int host_guard(F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return fail(HOBI_ERR_NOMEM, "host memory allocation failed");
  } catch (...) {
    return fail(HOBI_ERR_CUDA, "unexpected host-side exception");
  }
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (dev != prev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Analytic FP32 far-field block shape for a problem size (hobi_capi.cu).
int choose_shape(int n_targets, int n_pad, int num_sms);

// Device memory of the single-molecule handles comes from one library-owned stream-ordered pool
// per device (cudaMemPoolCreate, no release threshold): a handle set up after another one has
// been destroyed reuses the memory it returned instead of paying a cudaMalloc per table and a
// device-synchronising cudaFree per table at destruction. The pool keeps what it holds until the
// process exits. Allocations and frees are ordered on the handle's stream (hobi_capi.cu).
cudaError_t pool_alloc(void** p, size_t bytes, int device, cudaStream_t s);
cudaError_t pool_free(void* p, cudaStream_t s);

// The device buffers of one handle, or of a whole batch with its member handles. Buffers smaller
// than `direct` bytes are carved (256-byte aligned) from blocks of `chunk` bytes; larger ones get
// a block of their own. Every block is one stream-ordered allocation from the pool above, so a
// handle makes a few pool calls instead of one per table: once the pool holds thousands of freed
// blocks each call costs about 0.1 ms on the host (measured on GB300 with 64-molecule batches).
// A carved buffer is returned with the whole arena; put() returns an own-block buffer at once.
// A shared arena (a batch's, used by its members' streams from several host threads) locks, and
// allocates its blocks on the `home` stream and waits for them, so every block is ready for use
// on any stream.
struct DeviceArena {
  int device = 0;
  size_t chunk = size_t(4) << 20, direct = size_t(1) << 20;
  bool shared = false;
  cudaStream_t home = nullptr;
  std::mutex mu;
  std::vector<void*> chunks, own;  // carved-from blocks; buffers with a block of their own
  char* cur = nullptr;
  size_t left = 0;
  cudaError_t get(void** p, size_t bytes, cudaStream_t s);
  void put(void* p, cudaStream_t s);
  void release_all(cudaStream_t s);
};
// Pinned host slots of at most kPinnedSlot bytes (the GMRES state read-back, a host scalar) from
// a process-wide free list, pinned 64 at a time and kept until the process exits: a handle does
// not pay a cudaMallocHost / cudaFreeHost pair for them (hobi_capi.cu). nullptr on failure.
constexpr size_t kPinnedSlot = 256;
void* pinned_slot();
void pinned_slot_free(void* p);

}  // namespace host
}  // namespace hobi

#define HOBI_CK(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(HOBI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define HOBI_TRY(expr)        \
  do {                        \
    int r_ = (expr);          \
    if (r_ != HOBI_OK) return r_; \
  } while (0)

using namespace hobi;
using namespace hobi::host;

struct hobi_ctx {
  int device = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  int mem_device = 0, precision = HOBI_FP32_BULK, restart = 50, use_graph = 1, scheme = HOBI_SCHEME_HOBI;
  int autotune = 1, tuned = 0, ff_shape = -1;
  // nv: collocation points (mesh vertices for HOBI, face centroids for LOBI); nv_mesh: mesh vertices
  int64_t nv = 0, nf = 0, nc = 0, n_nodes = 0, n_pad = 0, nv_mesh = 0;
  int* zero_ptr = nullptr;  // LOBI: an all-zero incidence row pointer (no singular correction)
  int* ff_err = nullptr;    // far-field tile pipeline timeout flag (device)
  double eps1 = 1, eps2 = 80, kappa = 0, eps = 80;
  double xs = 1;            // coordinate scale of the far-field tables (ff32_coord_scale(kappa))
  int num_sms = 1;
  // fast summation (treecode) of the FP32 far field; fast_degree 0: direct summation
  int fast_degree = 0, fast_chunks = 1, fast_ntasks = 0, fast_nup = 0, fast_npc = 0, fast_resident = 1;
  int fast_batches = 0, fast_nseg = 0;
  double fast_theta = 0.7;
  int64_t fast_direct_pairs = 0, fast_approx_pairs = 0;
  int *fast_pos = nullptr, *fast_tmap = nullptr, *fast_pcoff = nullptr;
  int2 *fast_batch = nullptr, *fast_seg = nullptr, *fast_pcitems = nullptr;
  FastTask* fast_tasks = nullptr;
  FastUpItem* fast_up = nullptr;
  float *fast_axes = nullptr, *fast_half = nullptr;
  float4 *fast_src = nullptr, *fast_tgt = nullptr, *fast_partial = nullptr;
  // mixed-precision refinement (hobi_solve_refined): accumulated solution, residual, correction
  double *ref_x = nullptr, *ref_r = nullptr, *ref_d = nullptr, *ref_scal = nullptr;
  cudaEvent_t ref_t0 = nullptr, ref_t1 = nullptr;
  std::vector<FastTask> fast_tasks_h;  // host copies, for a batch that merges this molecule's plan
  std::vector<FastUpItem> fast_up_h;
  std::vector<int64_t> fast_task_cost_h;  // source entries of each task
  DeviceArena own_arena;
  DeviceArena* arena = &own_arena;  // a batch member carves its tables from the batch's arena
  // inputs and geometry
  double *V = nullptr, *Nin = nullptr, *Nv = nullptr, *Q = nullptr;
  int *F = nullptr, *deg = nullptr, *inc_ptr = nullptr, *inc_face = nullptr, *entry_vertex = nullptr;
  double *elem = nullptr, *ny = nullptr, *nnu = nullptr, *nW = nullptr, *corr = nullptr, *b = nullptr;
  double *center = nullptr, *vol_part = nullptr, *center_part = nullptr;
  int* flags = nullptr;
  float4 *tgt32 = nullptr, *ctgt32 = nullptr, *src32 = nullptr, *ptgt32 = nullptr;
  double *tgt64 = nullptr, *ctgt64 = nullptr, *src64 = nullptr, *ptgt64 = nullptr;
  double *part = nullptr, *ppart = nullptr, *phi_pts = nullptr, *pts_in = nullptr, *fld_pts = nullptr;
  size_t ppart_elems = 0, pts_cap = 0;
  FarFieldPlan plan[2];  // [0] FP64, [1] FP32 -- collocation-point targets, both rows
  // iterate vectors
  double *u_stage = nullptr, *au_stage = nullptr, *x = nullptr, *e_dev = nullptr;
  bool have_solution = false;
  // GMRES
  double *Vb = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *w = nullptr;
  double *hcol = nullptr, *cvec = nullptr, *dpart = nullptr, *nrm = nullptr;
  GmresState* st = nullptr;
  GmresState* st_host = nullptr;  // pinned
  double* host_scalar = nullptr;  // pinned
  // captured GMRES iteration per [precision][profiling]; the profiling variant carries event
  // record nodes around the far-field launch (gev), read after every replay
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaEvent_t gev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  double graph_pairs[2] = {0.0, 0.0};
  bool replay_prof_pending = false;
  bool graph_timing_unavailable = false;  // set if events inside graphs cannot be timed
  int replay_prof_pi = 0;
  // profiling of the far-field kernel
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
  size_t prof_used = 0;
  double prof_ms = 0.0, prof_pairs = 0.0;
  int64_t prof_launches = 0;
  double pending_pairs = 0.0;
  int64_t launches = 0;  // kernels this handle launched (graph replays count their kernels)
  bool capturing = false;
  // kernels in one GMRES iteration: gather, far field, combine, 2 x (dots, reduce, axpy),
  // norm dots + reduce, Givens, next basis vector, advance
  static constexpr int kIterationKernels = 14;
  int gmres_scaling = 1;        // GMRES on the unknowns scaled by D^-1 (hobi_options.gmres_scaling)
  double* dscale = nullptr;     // [2 n_v] the scale factor of each unknown (gmres_scaling)
  double* zvec = nullptr;       // [2 n_v] D^-1 times the current Arnoldi vector

  template <class T>
  int alloc(T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = arena->get(&q, bytes, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(HOBI_ERR_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                      cudaGetErrorString(e));
    }
    *p = static_cast<T*>(q);
    return HOBI_OK;
  }

  void release(void* p) { arena->put(p, stream); }

  // enter: work on the internal stream starts after everything already queued on the user stream
  int enter() {
    HOBI_CK(cudaEventRecord(ev_in, user_stream));
    HOBI_CK(cudaStreamWaitEvent(stream, ev_in, 0));
    return HOBI_OK;
  }
  // leave: the user stream continues after the internal work
  int leave() {
    HOBI_CK(cudaEventRecord(ev_out, stream));
    HOBI_CK(cudaStreamWaitEvent(user_stream, ev_out, 0));
    return HOBI_OK;
  }

  int copy_in(double* dst, const double* src, size_t count) {
    HOBI_CK(cudaMemcpyAsync(dst, src, count * sizeof(double),
                            mem_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream));
    return HOBI_OK;
  }
  int copy_out(double* dst, const double* src, size_t count) {
    HOBI_CK(cudaMemcpyAsync(dst, src, count * sizeof(double),
                            mem_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
    return HOBI_OK;
  }
  int finish() {
    HOBI_TRY(leave());
    if (!mem_device) HOBI_CK(cudaStreamSynchronize(stream));
    return HOBI_OK;
  }
  // A far-field tile pipeline that timed out leaves the result incomplete: report it.
  int check_farfield() {
    int flag = 0;
    HOBI_CK(cudaMemcpyAsync(&flag, ff_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    HOBI_CK(cudaStreamSynchronize(stream));
    if (flag) {
      HOBI_CK(cudaMemsetAsync(ff_err, 0, sizeof(int), stream));
      return fail(HOBI_ERR_CUDA, "far-field source-tile pipeline timed out (a bulk copy did not complete)");
    }
    return HOBI_OK;
  }

  // --------------------------------------------------------------- matvec pipeline
  bool fast_active(bool fp32) const { return fp32 && fast_degree > 0; }
  // one far-field evaluation: the planned direct kernel, or (fast) the treecode's proxy densities
  // and its list evaluation into the fast_chunks partial rows
  int launch_ff(bool fp32, bool fast, const FarFieldPlan& p, const float4* t32, const double* t64, double* out,
                bool skip_self) {
    if (!fast) {
      HOBI_CK(launch_farfield(fp32, p, t32, t64, src32, src64, eps, kappa, out, ff_err, stream, skip_self));
      return HOBI_OK;
    }
    HOBI_CK(launch_fast_upward(fast_nup, fast_up, fast_axes, fast_half, fast_src, fast_degree, fast_partial, fast_npc,
                               fast_pcitems, fast_pcoff, eps, stream));
    HOBI_CK(launch_fast_eval(fast_tasks, fast_ntasks, fast_batch, fast_seg, fast_src, fast_tgt, fast_tmap, (int)nv,
                             eps, kappa, out, ff_err, stream));
    return HOBI_OK;
  }
  int farfield(bool fp32, const FarFieldPlan& p, const float4* t32, const double* t64, double* out,
               bool skip_self = false, bool fast = false) {
    const double pairs = fast ? (double)(fast_direct_pairs + fast_approx_pairs) : (double)p.n_targets * (double)n_nodes;
    cudaEvent_t a = nullptr, bb = nullptr;
    if (prof && capturing) {
      const int pi = fp32 ? 1 : 0;
      for (int q = 0; q < 2; ++q)
        if (!gev[pi][q]) HOBI_CK(cudaEventCreate(&gev[pi][q]));
      HOBI_CK(cudaEventRecordWithFlags(gev[pi][0], stream, cudaEventRecordExternal));
      HOBI_TRY(launch_ff(fp32, fast, p, t32, t64, out, skip_self));
      HOBI_CK(cudaEventRecordWithFlags(gev[pi][1], stream, cudaEventRecordExternal));
      graph_pairs[pi] = pairs;
      return HOBI_OK;
    }
    if (prof) {
      if (prof_used == prof_ev.size()) {
        cudaEvent_t e0, e1;
        HOBI_CK(cudaEventCreate(&e0));
        HOBI_CK(cudaEventCreate(&e1));
        prof_ev.emplace_back(e0, e1);
      }
      a = prof_ev[prof_used].first;
      bb = prof_ev[prof_used].second;
      ++prof_used;
      HOBI_CK(cudaEventRecord(a, stream));
    }
    HOBI_TRY(launch_ff(fp32, fast, p, t32, t64, out, skip_self));
    if (prof) {
      HOBI_CK(cudaEventRecord(bb, stream));
      pending_pairs += pairs;
    }
    return HOBI_OK;
  }

  // node densities of u (scheme-dependent node layout)
  int gather(bool fp32, const double* u, const int* kptr, int64_t ld, bool fast = false) {
    if (scheme == HOBI_SCHEME_LOBI)
      HOBI_CK(launch_gather_lobi(fp32, (int)nf, ny, nnu, nW, center, u, kptr, ld, 1.0 / eps, xs, src32, src64,
                                 stream));
    else if (fast)  // tree order, into the treecode's source entries
      HOBI_CK(launch_gather(true, (int)n_nodes, (int)nv, F, ny, nnu, nW, center, u, kptr, ld, 1.0 / eps, xs,
                            fast_src, src64, stream, fast_pos));
    else
      HOBI_CK(launch_gather(fp32, (int)n_nodes, (int)nv, F, ny, nnu, nW, center, u, kptr, ld, 1.0 / eps, xs,
                            src32, src64, stream));
    return HOBI_OK;
  }

  template <class T>
  int upload(T** dev, const std::vector<T>& v) {
    HOBI_TRY(alloc(dev, v.size()));
    if (!v.empty()) HOBI_CK(cudaMemcpyAsync(*dev, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, stream));
    return HOBI_OK;
  }
  // Treecode plan (host) from the FP64 node and vertex coordinates, uploaded with its buffers.
  // piece_sources > 0: evaluation pieces of about that many source entries (batch use).
  int setup_fast(int piece_sources = 0) {
    std::vector<double> hy(3 * (size_t)n_nodes), hx(3 * (size_t)nv), hc(3);
    HOBI_CK(cudaMemcpyAsync(hy.data(), ny, sizeof(double) * hy.size(), cudaMemcpyDeviceToHost, stream));
    HOBI_CK(cudaMemcpyAsync(hx.data(), V, sizeof(double) * hx.size(), cudaMemcpyDeviceToHost, stream));
    HOBI_CK(cudaMemcpyAsync(hc.data(), center, sizeof(double) * 3, cudaMemcpyDeviceToHost, stream));
    HOBI_CK(cudaStreamSynchronize(stream));
    fast_resident = num_sms * fast_eval_blocks_per_sm(kappa);  // evaluation blocks resident at once
    FastPlanHost P;
    build_fast_plan(hy.data(), (int)n_nodes, hx.data(), (int)nv, hc.data(), xs, fast_degree, fast_theta, fast_resident,
                    piece_sources, &P);
    const int n3 = (fast_degree + 1) * (fast_degree + 1) * (fast_degree + 1);
    fast_chunks = P.chunks;
    fast_ntasks = (int)P.tasks.size();
    fast_nup = (int)P.up.size();
    fast_npc = (int)P.pc_offset.size();
    fast_batches = (int)P.batch.size();
    fast_nseg = (int)P.seg.size();
    fast_direct_pairs = P.direct_pairs;
    fast_approx_pairs = P.approx_pairs;
    fast_tasks_h = P.tasks;
    fast_up_h = P.up;
    fast_task_cost_h.clear();
    for (const FastTask& t : P.tasks) {
      int64_t c = 0;
      for (int q = t.s0; q < t.s1; ++q) c += P.seg[q].y;
      fast_task_cost_h.push_back(c);
    }
    HOBI_TRY(upload(&fast_pos, P.node_pos));
    HOBI_TRY(upload(&fast_tmap, P.tmap));
    HOBI_TRY(upload(&fast_batch, P.batch));
    HOBI_TRY(upload(&fast_seg, P.seg));
    HOBI_TRY(upload(&fast_tasks, P.tasks));
    HOBI_TRY(upload(&fast_up, P.up));
    HOBI_TRY(upload(&fast_pcitems, P.pc_items));
    HOBI_TRY(upload(&fast_pcoff, P.pc_offset));
    HOBI_TRY(upload(&fast_axes, P.axes));
    HOBI_TRY(upload(&fast_half, P.half));
    HOBI_TRY(alloc(&fast_src, 4 * (size_t)P.n_entries));
    HOBI_TRY(alloc(&fast_tgt, 2 * (size_t)nv));
    HOBI_TRY(alloc(&fast_partial, (size_t)fast_nup * n3));
    HOBI_CK(launch_fast_targets((int)nv, fast_tmap, tgt32, fast_tgt, stream));
    launches += 1;
    HOBI_CK(cudaStreamSynchronize(stream));  // the host vectors above are released on return
    return HOBI_OK;
  }

  // Au = A u with u = base + (*kptr) * ld when kptr is given (device pointers)
  int matvec_dev(const double* u, const int* kptr, int64_t ld, double* Au) {
    const bool fp32 = precision == HOBI_FP32_BULK;
    const bool lobi = scheme == HOBI_SCHEME_LOBI;
    const bool fast = fast_active(fp32);
    HOBI_TRY(gather(fp32, u, kptr, ld, fast));
    HOBI_TRY(farfield(fp32, plan[fp32], tgt32, tgt64, part, lobi, fast));
    HOBI_CK(launch_combine((int)nv, fast ? fast_chunks : plan[fp32].chunks, part, F, lobi ? zero_ptr : inc_ptr,
                           inc_face, corr, eps, u, kptr, ld, Au, stream));
    if (!capturing) launches += fast ? 5 : 3;
    return HOBI_OK;
  }

  int collect_profile() {
    if (!prof || prof_used == 0) return HOBI_OK;
    HOBI_CK(cudaStreamSynchronize(stream));
    for (size_t i = 0; i < prof_used; ++i) {
      float ms = 0.f;
      HOBI_CK(cudaEventElapsedTime(&ms, prof_ev[i].first, prof_ev[i].second));
      prof_ms += ms;
    }
    prof_launches += (int64_t)prof_used;
    prof_pairs += pending_pairs;
    pending_pairs = 0.0;
    prof_used = 0;
    return HOBI_OK;
  }

  // --------------------------------------------------------------- GMRES iteration body
  int iteration() {
    const int64_t n = 2 * nv;
    const int m = restart;
    if (gmres_scaling) {  // w = A D^-1 v_k (right preconditioning by the constant diagonal)
      HOBI_CK(launch_scale_column(Vb, n, &st->k, dscale, zvec, n, stream));
      if (!capturing) launches += 1;
      HOBI_TRY(matvec_dev(zvec, nullptr, 0, w));
    } else {
      HOBI_TRY(matvec_dev(Vb, &st->k, n, w));
    }
    for (int pass = 0; pass < 2; ++pass) {
      HOBI_CK(launch_dots(Vb, n, w, n, st, 0, dpart, stream));
      HOBI_CK(launch_reduce_dots(dpart, m, st, 0, cvec, hcol, pass, stream));
      HOBI_CK(launch_axpy_basis(Vb, n, cvec, st, w, n, stream));
    }
    HOBI_CK(launch_dots(nullptr, 0, w, n, st, 1, dpart, stream));
    HOBI_CK(launch_reduce_dots(dpart, m, st, 1, nrm, nullptr, 0, stream));
    HOBI_CK(launch_givens(st, m, H, cs, sn, g, hcol, nrm, stream));
    HOBI_CK(launch_next_basis(Vb, n, w, n, st, stream));
    HOBI_CK(launch_advance(st, stream));
    if (!capturing) launches += kIterationKernels - 3;
    return HOBI_OK;
  }

  int run_iteration() {
    const int pi = precision == HOBI_FP32_BULK;
    if (!use_graph || (prof && graph_timing_unavailable)) return iteration();
    cudaGraphExec_t& gx = graph[pi][prof ? 1 : 0];
    if (!gx) {
      cudaGraph_t gr = nullptr;
      HOBI_CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
      capturing = true;
      int r = iteration();
      capturing = false;
      cudaError_t e = cudaStreamEndCapture(stream, &gr);
      if (r != HOBI_OK) {
        if (gr) cudaGraphDestroy(gr);
        return r;
      }
      if (e != cudaSuccess) return fail(HOBI_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&gx, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) {
        gx = nullptr;
        return fail(HOBI_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      }
    }
    HOBI_CK(cudaGraphLaunch(gx, stream));
    launches += kIterationKernels + (fast_active(pi) ? 2 : 0) + (gmres_scaling ? 1 : 0);
    if (prof) {
      replay_prof_pending = true;
      replay_prof_pi = pi;
    }
    return HOBI_OK;
  }

  int read_state() {
    HOBI_CK(cudaMemcpyAsync(st_host, st, sizeof(GmresState), cudaMemcpyDeviceToHost, stream));
    HOBI_CK(cudaStreamSynchronize(stream));
    if (replay_prof_pending) {  // far-field time inside the graph that just completed
      float ms = 0.f;
      replay_prof_pending = false;
      if (cudaEventElapsedTime(&ms, gev[replay_prof_pi][0], gev[replay_prof_pi][1]) != cudaSuccess) {
        cudaGetLastError();
        graph_timing_unavailable = true;  // later profiled iterations launch directly
      } else {
        prof_ms += ms;
        prof_launches += 1;
        prof_pairs += graph_pairs[replay_prof_pi];
      }
    }
    return HOBI_OK;
  }

  // Point buffers grow at least geometrically: a carved buffer that is outgrown stays in the
  // arena until the handle is destroyed, so the held memory stays below twice the largest need.
  int ensure_point_buffers(int64_t np) {
    if ((size_t)np <= pts_cap) return HOBI_OK;
    const size_t cap = std::max<size_t>({(size_t)64, (size_t)np, 2 * pts_cap});
    if (ptgt32) { release(ptgt32); release(ptgt64); release(phi_pts); release(pts_in); release(fld_pts); }
    HOBI_TRY(alloc(&ptgt32, 2 * cap));
    HOBI_TRY(alloc(&ptgt64, 8 * cap));
    HOBI_TRY(alloc(&phi_pts, cap));
    HOBI_TRY(alloc(&pts_in, 3 * cap));
    HOBI_TRY(alloc(&fld_pts, 3 * cap));
    pts_cap = cap;
    return HOBI_OK;
  }
  int ensure_ppart(size_t elems) {
    if (elems <= ppart_elems) return HOBI_OK;
    elems = std::max(elems, 2 * ppart_elems);
    if (ppart) release(ppart);
    HOBI_TRY(alloc(&ppart, elems));
    ppart_elems = elems;
    return HOBI_OK;
  }

  // -grad phi_reac at np targets already in (t32, t64), [np][3], from the current solution x
  int field_dev(int64_t np, const float4* t32, const double* t64, double* field) {
    const bool fp32 = precision == HOBI_FP32_BULK;
    FarFieldPlan p = plan_farfield(fp32, (int)np, (int)n_pad, false, num_sms, field_blocks_per_sm(fp32, kappa), 0);
    HOBI_TRY(ensure_ppart((size_t)p.chunks * 3 * (size_t)np));
    HOBI_TRY(gather(fp32, x, nullptr, 0));
    HOBI_CK(launch_field(fp32, p, t32, t64, src32, src64, eps, kappa, ppart, ff_err, stream));
    HOBI_CK(launch_reduce_field((int)np, p.chunks, ppart, field, stream));
    launches += 3;
    return HOBI_OK;
  }

  // phi_reac at np targets already in (t32, t64), row 1 only, from the current solution x
  int reaction_dev(int64_t np, const float4* t32, const double* t64, double* phi) {
    const bool fp32 = precision == HOBI_FP32_BULK;
    const int sh = fp32 ? choose_shape((int)np, (int)n_pad, num_sms) : 0;
    FarFieldPlan p = plan_farfield(fp32, (int)np, (int)n_pad, false, num_sms, farfield_blocks_per_sm(fp32, false, sh), sh);
    HOBI_TRY(ensure_ppart((size_t)p.chunks * (size_t)np));
    HOBI_TRY(gather(fp32, x, nullptr, 0));
    HOBI_TRY(farfield(fp32, p, t32, t64, ppart));
    HOBI_CK(launch_reduce_points((int)np, p.chunks, ppart, phi, stream));
    launches += 3;
    return HOBI_OK;
  }

  ~hobi_ctx() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto& row : graph)
      for (auto& gexec : row)
        if (gexec) cudaGraphExecDestroy(gexec);
    for (auto& row : gev)
      for (auto& ev : row)
        if (ev) cudaEventDestroy(ev);
    own_arena.release_all(stream);
    for (auto& e : prof_ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    if (st_host) pinned_slot_free(st_host);
    if (host_scalar) pinned_slot_free(host_scalar);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (ev_t0) cudaEventDestroy(ev_t0);
    if (ev_t1) cudaEventDestroy(ev_t1);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace hobi {
namespace host {
// Validates the inputs, copies them to the device and builds every table of one molecule
// (hobi_setup); light = 1 skips the per-molecule Krylov workspace and graphs (batch members).
// A non-null arena (a batch's) holds the handle's device buffers instead of its own arena; it
// must outlive the handle.
int create_handle(const double* vertices, int64_t n_v, const int32_t* faces, int64_t n_f, const double* vertex_normals,
                  const double* charges, int64_t n_c, double eps1, double eps2, double kappa, const hobi_options* opt,
                  bool light, hobi_t* out, DeviceArena* arena = nullptr);
// hobi_energy in two parts: queue the work on the handle's stream, then wait and read E_sol.
int energy_enqueue(hobi_ctx* h);
int energy_finish(hobi_ctx* h, double* e_sol);
}  // namespace host
}  // namespace hobi
