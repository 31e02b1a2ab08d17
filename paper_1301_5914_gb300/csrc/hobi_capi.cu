// hobi_capi.cu -- the C ABI declared in include/hobi.h: handle lifetime, device memory, stream
// ordering, the setup pipeline, the matvec pipeline, the GMRES driver (optionally replayed from a
// captured CUDA graph) and the energy.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <stdio.h>
#include <stdlib.h>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hobi.h"
#include "hobi_internal.cuh"

namespace {
// NVTX range around a public call (no-op unless a profiler is attached), so nsys / ncu timelines
// show setup, matvec, solve and energy phases by name.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

using namespace hobi;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

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

int choose_shape(int n_targets, int n_pad, int num_sms);

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

}  // namespace

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
  std::vector<void*> allocs;
  // inputs and geometry
  double *V = nullptr, *Nin = nullptr, *Nv = nullptr, *Q = nullptr;
  int *F = nullptr, *deg = nullptr, *inc_ptr = nullptr, *inc_face = nullptr, *entry_vertex = nullptr;
  double *elem = nullptr, *ny = nullptr, *nnu = nullptr, *nW = nullptr, *corr = nullptr, *b = nullptr;
  double *center = nullptr, *vol_part = nullptr, *center_part = nullptr;
  int* flags = nullptr;
  float4 *tgt32 = nullptr, *ctgt32 = nullptr, *src32 = nullptr, *ptgt32 = nullptr;
  double *tgt64 = nullptr, *ctgt64 = nullptr, *src64 = nullptr, *ptgt64 = nullptr;
  double *part = nullptr, *ppart = nullptr, *phi_pts = nullptr, *pts_in = nullptr;
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

  template <class T>
  int alloc(T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(HOBI_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                      cudaGetErrorString(e));
    }
    allocs.push_back(q);
    *p = static_cast<T*>(q);
    return HOBI_OK;
  }

  void release(void* p) {
    for (auto& a : allocs)
      if (a == p) {
        cudaFree(a);
        a = nullptr;
      }
  }

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
    HOBI_TRY(matvec_dev(Vb, &st->k, n, w));
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
    launches += kIterationKernels + (fast_active(pi) ? 2 : 0);
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

  int ensure_point_buffers(int64_t np) {
    if ((size_t)np <= pts_cap) return HOBI_OK;
    size_t cap = (size_t)np < 64 ? 64 : (size_t)np;
    if (ptgt32) { release(ptgt32); release(ptgt64); release(phi_pts); release(pts_in); }
    HOBI_TRY(alloc(&ptgt32, 2 * cap));
    HOBI_TRY(alloc(&ptgt64, 8 * cap));
    HOBI_TRY(alloc(&phi_pts, cap));
    HOBI_TRY(alloc(&pts_in, 3 * cap));
    pts_cap = cap;
    return HOBI_OK;
  }
  int ensure_ppart(size_t elems) {
    if (elems <= ppart_elems) return HOBI_OK;
    if (ppart) release(ppart);
    HOBI_TRY(alloc(&ppart, elems));
    ppart_elems = elems;
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
    for (void* p : allocs)
      if (p) cudaFree(p);
    for (auto& e : prof_ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    if (st_host) cudaFreeHost(st_host);
    if (host_scalar) cudaFreeHost(host_scalar);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (ev_t0) cudaEventDestroy(ev_t0);
    if (ev_t1) cudaEventDestroy(ev_t1);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

// Analytic shape choice: the largest block shape that still yields enough independent
// (target block, source tile) work items to fill the machine several times over.
int choose_shape(int n_targets, int n_pad, int num_sms) {
  static const int per_block[kNumFF32Shapes] = {256, 512, 256, 128};
  static const int tile[kNumFF32Shapes] = {128, 128, 64, 64};
  for (int s = 0; s < kNumFF32Shapes; ++s) {
    long tt = (n_targets + per_block[s] - 1) / per_block[s];
    long tiles = n_pad / tile[s];
    if (tt * std::min<long>(tiles, 512) >= 8L * num_sms * farfield_blocks_per_sm(true, true, s)) return s;
  }
  return kNumFF32Shapes - 1;
}

constexpr int kTuneLaunches = 4;  // per candidate shape: one warm-up, then the fastest of three

// Autotuner decisions, per process (and optionally in a file): key -> shape
std::mutex g_tune_mu;
std::vector<std::pair<std::string, int>> g_tune;
bool g_tune_loaded = false;

std::string tune_key(int device, int scheme, int64_t nv, int64_t n_pad) {
  cudaDeviceProp prop;
  std::string name = cudaGetDeviceProperties(&prop, device) == cudaSuccess ? prop.name : "gpu";
  for (char& c : name)
    if (c == ' ') c = '_';
  return name + " " + std::to_string(scheme) + " " + std::to_string(nv) + " " + std::to_string(n_pad);
}

bool tune_lookup(const std::string& key, int* shape) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (!g_tune_loaded) {
    g_tune_loaded = true;
    if (const char* path = getenv("HOBI_AUTOTUNE_CACHE")) {
      if (FILE* f = fopen(path, "r")) {
        char a[256], b[32], c[32], d[32];
        int sh;
        while (fscanf(f, "%255s %31s %31s %31s %d", a, b, c, d, &sh) == 5)
          if (sh >= 0 && sh < kNumFF32Shapes)
            g_tune.emplace_back(std::string(a) + " " + b + " " + c + " " + d, sh);
        fclose(f);
      }
    }
  }
  for (auto& kv : g_tune)
    if (kv.first == key) {
      *shape = kv.second;
      return true;
    }
  return false;
}

void tune_store(const std::string& key, int shape) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.emplace_back(key, shape);
  if (const char* path = getenv("HOBI_AUTOTUNE_CACHE")) {
    if (FILE* f = fopen(path, "a")) {
      fprintf(f, "%s %d\n", key.c_str(), shape);
      fclose(f);
    }
  }
}

std::string mesh_message(int fl) {
  std::string m = "invalid mesh:";
  if (fl & kBadIndex) m += " face index out of range or repeated within a face;";
  if (fl & kOpenOrInconsistent) m += " surface not closed or not consistently oriented (a directed edge lacks exactly one opposite edge);";
  if (fl & kUnreferencedVertex) m += " vertex referenced by no face;";
  if (fl & kBadNormal) m += " zero or non-finite vertex normal;";
  if (fl & kNonFinite) m += " non-finite vertex coordinate;";
  if (fl & kNegativeVolume) m += " enclosed volume not positive (faces must be counter-clockwise seen from outside);";
  if (fl & kDegenerateFace) m += " zero-area face;";
  if (fl & kBadCharge) m += " non-finite charge;";
  return m;
}

// light: a member of a batch -- tables only; the batch owns partial sums and Krylov workspace
int setup_impl(hobi_ctx* h, const double* vertices, const int32_t* faces, const double* normals,
               const double* charges, bool light) {
  const int64_t nv = h->nv, nf = h->nf, nc = h->nc;
  const cudaMemcpyKind kind = h->mem_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  HOBI_TRY(h->alloc(&h->V, 3 * nv));
  HOBI_TRY(h->alloc(&h->Nin, 3 * nv));
  HOBI_TRY(h->alloc(&h->Nv, 3 * nv));
  HOBI_TRY(h->alloc(&h->F, 3 * nf));
  HOBI_TRY(h->alloc(&h->Q, 4 * (nc > 0 ? nc : 1)));
  HOBI_TRY(h->alloc(&h->deg, nv));
  HOBI_TRY(h->alloc(&h->inc_ptr, nv + 1));
  HOBI_TRY(h->alloc(&h->inc_face, 3 * nf));
  HOBI_TRY(h->alloc(&h->entry_vertex, 3 * nf));
  HOBI_TRY(h->alloc(&h->vol_part, kValidateBlocks));
  HOBI_TRY(h->alloc(&h->center_part, 3 * kValidateBlocks));
  HOBI_TRY(h->alloc(&h->center, 3));
  HOBI_TRY(h->alloc(&h->flags, 1));
  HOBI_TRY(h->alloc(&h->ff_err, 1));
  HOBI_CK(cudaMemsetAsync(h->ff_err, 0, sizeof(int), h->stream));
  HOBI_CK(cudaMemcpyAsync(h->V, vertices, sizeof(double) * 3 * nv, kind, h->stream));
  HOBI_CK(cudaMemcpyAsync(h->Nin, normals, sizeof(double) * 3 * nv, kind, h->stream));
  HOBI_CK(cudaMemcpyAsync(h->F, faces, sizeof(int32_t) * 3 * nf, kind, h->stream));
  if (nc > 0) HOBI_CK(cudaMemcpyAsync(h->Q, charges, sizeof(double) * 4 * nc, kind, h->stream));
  HOBI_CK(cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream));

  // adjacency and validation
  HOBI_CK(launch_adjacency((int)nv, (int)nf, h->F, h->deg, h->inc_ptr, h->inc_face, h->entry_vertex, h->stream));
  HOBI_CK(launch_validate((int)nv, (int)nf, (int)nc, h->V, h->Nin, h->F, h->inc_ptr, h->inc_face, h->Q, h->Nv,
                          h->vol_part, h->center_part, h->flags, h->stream));
  HOBI_CK(launch_finish_validate((int)nv, h->vol_part, h->center_part, h->center, h->flags, h->stream));
  h->launches += 5 + 3 + (nc > 0 ? 1 : 0);  // adjacency (5), validation (3 + charges)
  int flags = 0;
  HOBI_CK(cudaMemcpyAsync(&flags, h->flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HOBI_CK(cudaStreamSynchronize(h->stream));
  if (flags == kBadCharge) return fail(HOBI_ERR_ARG, "non-finite charge position or value");
  if (flags) return fail(HOBI_ERR_MESH, mesh_message(flags));

  h->nv_mesh = nv;
  if (h->scheme == HOBI_SCHEME_LOBI) {
    // LOBI-PB (Sec. 2.4): one node per flat face at its centroid; collocation at the centroids
    h->nv = nf;
    h->n_nodes = nf;
    h->n_pad = (h->n_nodes + kTile - 1) / kTile * kTile;
    HOBI_TRY(h->alloc(&h->ny, 3 * nf));
    HOBI_TRY(h->alloc(&h->nnu, 3 * nf));
    HOBI_TRY(h->alloc(&h->nW, 3 * nf));
    HOBI_TRY(h->alloc(&h->zero_ptr, nf + 1));
    HOBI_TRY(h->alloc(&h->b, 2 * nf));
    HOBI_TRY(h->alloc(&h->tgt32, 2 * nf));
    HOBI_TRY(h->alloc(&h->tgt64, 8 * nf));
    HOBI_TRY(h->alloc(&h->ctgt32, 2 * (nc > 0 ? nc : 1)));
    HOBI_TRY(h->alloc(&h->ctgt64, 8 * (nc > 0 ? nc : 1)));
    HOBI_TRY(h->alloc(&h->src32, 4 * h->n_pad));
    HOBI_TRY(h->alloc(&h->src64, 8 * h->n_pad));
    HOBI_CK(cudaMemsetAsync(h->zero_ptr, 0, sizeof(int) * (nf + 1), h->stream));
    HOBI_CK(launch_lobi_geometry((int)nf, h->F, h->V, h->ny, h->nnu, h->nW, h->flags, h->stream));
    HOBI_CK(launch_rhs((int)nf, (int)nc, h->ny, h->nnu, h->Q, h->eps1, h->b, h->stream));
    HOBI_CK(launch_targets((int)nf, h->ny, h->nnu, h->center, h->xs, h->tgt32, h->tgt64, h->stream));
    HOBI_CK(launch_points((int)nc, h->Q, 4, h->center, h->xs, h->ctgt32, h->ctgt64, h->stream));
    HOBI_CK(launch_pad_sources((int)h->n_nodes, (int)h->n_pad, h->src32, h->src64, h->stream));
    h->launches += 3 + (nc > 0 ? 1 : 0) + (h->n_pad > h->n_nodes ? 1 : 0);
  } else {
    // curved elements, nodes, correction, right-hand side (Sec. 2.6 routines (1)-(4))
    h->n_nodes = 4 * nf;
    h->n_pad = (h->n_nodes + kTile - 1) / kTile * kTile;
    HOBI_TRY(h->alloc(&h->elem, 30 * nf));
    HOBI_TRY(h->alloc(&h->ny, 3 * h->n_nodes));
    HOBI_TRY(h->alloc(&h->nnu, 3 * h->n_nodes));
    HOBI_TRY(h->alloc(&h->nW, 3 * h->n_nodes));
    HOBI_TRY(h->alloc(&h->corr, 12 * 3 * nf));
    HOBI_TRY(h->alloc(&h->b, 2 * nv));
    HOBI_TRY(h->alloc(&h->tgt32, 2 * nv));
    HOBI_TRY(h->alloc(&h->tgt64, 8 * nv));
    HOBI_TRY(h->alloc(&h->ctgt32, 2 * (nc > 0 ? nc : 1)));
    HOBI_TRY(h->alloc(&h->ctgt64, 8 * (nc > 0 ? nc : 1)));
    HOBI_TRY(h->alloc(&h->src32, 4 * h->n_pad));
    HOBI_TRY(h->alloc(&h->src64, 8 * h->n_pad));
    HOBI_CK(launch_node_gen((int)nf, h->F, h->V, h->Nv, h->elem, h->ny, h->nnu, h->nW, h->flags, h->stream));
    HOBI_CK(launch_correction_entries((int)(3 * nf), h->entry_vertex, h->F, h->V, h->Nv, h->inc_face, h->elem, h->ny,
                                      h->nnu, h->nW, h->eps, h->kappa, h->corr, h->stream));
    HOBI_CK(launch_rhs((int)nv, (int)nc, h->V, h->Nv, h->Q, h->eps1, h->b, h->stream));
    HOBI_CK(launch_targets((int)nv, h->V, h->Nv, h->center, h->xs, h->tgt32, h->tgt64, h->stream));
    HOBI_CK(launch_points((int)nc, h->Q, 4, h->center, h->xs, h->ctgt32, h->ctgt64, h->stream));
    HOBI_CK(launch_pad_sources((int)h->n_nodes, (int)h->n_pad, h->src32, h->src64, h->stream));
    h->launches += 4 + (nc > 0 ? 1 : 0) + (h->n_pad > h->n_nodes ? 1 : 0);
  }
  HOBI_CK(cudaMemcpyAsync(&flags, h->flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HOBI_CK(cudaStreamSynchronize(h->stream));
  if (flags & kDegenerateElement)
    return fail(HOBI_ERR_MESH, "invalid mesh: a curved element has a zero or non-finite area Jacobian "
                               "(vertex normals inconsistent with the faces)");

  HOBI_TRY(h->alloc(&h->x, 2 * h->nv));
  HOBI_TRY(h->alloc(&h->e_dev, 1));
  HOBI_CK(cudaMallocHost(&h->host_scalar, sizeof(double)));
  if (light) {
    HOBI_CK(cudaStreamSynchronize(h->stream));
    return HOBI_OK;
  }
  // far-field plans and partial-sum buffers (room for every FP32 shape the autotuner may try)
  const bool skip = h->scheme == HOBI_SCHEME_LOBI;
  FarFieldPlan cand[kNumFF32Shapes];
  size_t part_elems = 0;
  for (int sh = 0; sh < kNumFF32Shapes; ++sh) {
    cand[sh] = plan_farfield(true, (int)h->nv, (int)h->n_pad, true, h->num_sms, farfield_blocks_per_sm(true, true, sh),
                             sh);
    part_elems = std::max(part_elems, (size_t)cand[sh].chunks * 2 * h->nv);
  }
  h->plan[0] = plan_farfield(false, (int)h->nv, (int)h->n_pad, true, h->num_sms, farfield_blocks_per_sm(false, true));
  part_elems = std::max(part_elems, (size_t)h->plan[0].chunks * 2 * h->nv);
  if (h->fast_degree > 0) {
    HOBI_TRY(h->setup_fast());
    part_elems = std::max(part_elems, (size_t)h->fast_chunks * 2 * h->nv);
  }
  HOBI_TRY(h->alloc(&h->part, part_elems));
  int shape = choose_shape((int)h->nv, (int)h->n_pad, h->num_sms);
  if (h->ff_shape >= 0) {
    shape = h->ff_shape;
  } else if (h->autotune && h->fast_degree == 0) {
    const std::string key = tune_key(h->device, h->scheme, h->nv, h->n_pad);
    if (tune_lookup(key, &shape)) {
      h->tuned = 1;
    } else {
      // time every shape on this problem (densities of u = 0; the timing does not depend on them)
      HOBI_CK(cudaMemsetAsync(h->x, 0, sizeof(double) * 2 * h->nv, h->stream));
      HOBI_TRY(h->gather(true, h->x, nullptr, 0));
      float best = 1e30f;
      for (int sh = 0; sh < kNumFF32Shapes; ++sh) {
        float t = 1e30f;
        for (int rep = 0; rep < kTuneLaunches; ++rep) {
          HOBI_CK(cudaEventRecord(h->ev_t0, h->stream));
          HOBI_CK(launch_farfield(true, cand[sh], h->tgt32, h->tgt64, h->src32, h->src64, h->eps, h->kappa, h->part,
                                  h->ff_err, h->stream, skip));
          HOBI_CK(cudaEventRecord(h->ev_t1, h->stream));
          HOBI_CK(cudaEventSynchronize(h->ev_t1));
          float ms = 0.f;
          HOBI_CK(cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1));
          if (rep > 0) t = std::min(t, ms);  // the first launch warms up; the fastest of the rest
        }
        h->launches += kTuneLaunches;
        if (t < best * 0.98f) {  // prefer the earlier (larger) shape unless clearly faster
          best = t;
          shape = sh;
        }
      }
      HOBI_TRY(h->check_farfield());
      tune_store(key, shape);
      h->tuned = 1;
    }
  }
  h->plan[1] = cand[shape];

  // iterate vectors and GMRES workspace
  const int64_t n = 2 * h->nv;
  const int m = h->restart;
  HOBI_TRY(h->alloc(&h->u_stage, n));
  HOBI_TRY(h->alloc(&h->au_stage, n));
  HOBI_TRY(h->alloc(&h->Vb, (size_t)(m + 1) * n));
  HOBI_TRY(h->alloc(&h->H, (size_t)(m + 1) * m));
  HOBI_TRY(h->alloc(&h->cs, m));
  HOBI_TRY(h->alloc(&h->sn, m));
  HOBI_TRY(h->alloc(&h->g, m + 1));
  HOBI_TRY(h->alloc(&h->y, m));
  HOBI_TRY(h->alloc(&h->w, n));
  HOBI_TRY(h->alloc(&h->hcol, m + 1));
  HOBI_TRY(h->alloc(&h->cvec, m + 1));
  HOBI_TRY(h->alloc(&h->nrm, 1));
  HOBI_TRY(h->alloc(&h->dpart, (size_t)(m + 1) * kDotBlocks));
  HOBI_TRY(h->alloc(&h->st, 1));
  HOBI_CK(cudaMallocHost(&h->st_host, sizeof(GmresState)));
  HOBI_CK(cudaMemsetAsync(h->H, 0, sizeof(double) * (m + 1) * m, h->stream));
  HOBI_CK(cudaStreamSynchronize(h->stream));
  return HOBI_OK;
}

}  // namespace

extern "C" {

void hobi_default_options(hobi_options* opt) {
  if (!opt) return;
  opt->precision = HOBI_FP32_BULK;
  opt->mem_device = 0;
  opt->stream = nullptr;
  opt->restart = 50;
  opt->use_graph = 1;
  opt->device = -1;
  opt->scheme = HOBI_SCHEME_HOBI;
  opt->autotune = 1;
  opt->ff_shape = -1;
  opt->fast_degree = 0;
  opt->fast_theta = 0.7;
}

const char* hobi_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace {
int create_handle(const double* vertices, int64_t n_v, const int32_t* faces, int64_t n_f, const double* vertex_normals,
                  const double* charges, int64_t n_c, double eps1, double eps2, double kappa, const hobi_options* opt,
                  bool light, hobi_t* out) {
  g_err.clear();
  if (!out) return fail(HOBI_ERR_ARG, "out handle pointer is NULL");
  *out = nullptr;
  if (!vertices || !faces || !vertex_normals)
    return fail(HOBI_ERR_ARG, "vertices, faces and vertex_normals must be non-NULL");
  if (n_c > 0 && !charges) return fail(HOBI_ERR_ARG, "charges is NULL but n_c > 0");
  if (n_v < 4 || n_f < 4) return fail(HOBI_ERR_ARG, "a closed surface needs at least 4 vertices and 4 faces");
  if (n_c < 0) return fail(HOBI_ERR_ARG, "n_c < 0");
  if (n_f > (int64_t(1) << 28) || n_v > (int64_t(1) << 28) || n_c > (int64_t(1) << 28))
    return fail(HOBI_ERR_ARG, "problem too large (n_v, n_f, n_c must be < 2^28)");
  if (!(eps1 > 0.0) || !(eps2 > 0.0) || !isfinite(eps1) || !isfinite(eps2))
    return fail(HOBI_ERR_ARG, "eps1 and eps2 must be finite and > 0");
  if (!(kappa >= 0.0) || !isfinite(kappa)) return fail(HOBI_ERR_ARG, "kappa must be finite and >= 0");
  hobi_options o;
  hobi_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != HOBI_FP64 && o.precision != HOBI_FP32_BULK) return fail(HOBI_ERR_ARG, "unknown precision");
  if (o.scheme != HOBI_SCHEME_HOBI && o.scheme != HOBI_SCHEME_LOBI) return fail(HOBI_ERR_ARG, "unknown scheme");
  if (o.ff_shape < -1 || o.ff_shape >= kNumFF32Shapes) return fail(HOBI_ERR_ARG, "ff_shape must be -1 or 0..3");
  if (o.fast_degree != 0 && (o.fast_degree < 2 || o.fast_degree > kFastMaxDegree))
    return fail(HOBI_ERR_ARG, "fast_degree must be 0 (direct far field) or 2..10");
  if (o.fast_degree != 0 && !(o.fast_theta > 0.0 && o.fast_theta <= 1.0))
    return fail(HOBI_ERR_ARG, "fast_theta must be in (0, 1]");
  if (o.fast_degree != 0 && o.scheme != HOBI_SCHEME_HOBI)
    return fail(HOBI_ERR_ARG, "fast summation is implemented for the HOBI scheme only");
  if (o.restart <= 0) o.restart = 50;
  if (o.restart > 200) return fail(HOBI_ERR_ARG, "restart must be <= 200");

  int dev = o.device;
  if (dev < 0) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HOBI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  DeviceGuard guard(dev);
  hobi_ctx* h = new hobi_ctx();
  h->device = dev;
  h->user_stream = static_cast<cudaStream_t>(o.stream);
  h->mem_device = o.mem_device ? 1 : 0;
  h->precision = o.precision;
  h->restart = o.restart;
  h->use_graph = o.use_graph ? 1 : 0;
  h->scheme = o.scheme;
  h->autotune = o.autotune ? 1 : 0;
  h->ff_shape = o.ff_shape;
  h->fast_degree = o.fast_degree;
  h->fast_theta = o.fast_theta;
  h->nv = n_v;
  h->nf = n_f;
  h->nc = n_c;
  h->eps1 = eps1;
  h->eps2 = eps2;
  h->kappa = kappa;
  h->xs = ff32_coord_scale(kappa);
  h->eps = eps2 / eps1;
  int r = HOBI_OK;
  do {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev_t0);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev_t1);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      r = fail(HOBI_ERR_CUDA, std::string("stream/event setup: ") + cudaGetErrorString(e));
      break;
    }
    r = h->enter();
    if (r != HOBI_OK) break;
    r = setup_impl(h, vertices, faces, vertex_normals, charges, light);
    if (r != HOBI_OK) break;
    r = h->leave();
  } while (0);
  if (r != HOBI_OK) {
    std::string msg = g_err;
    delete h;
    g_err = msg;
    return r;
  }
  *out = h;
  return HOBI_OK;
}
}  // namespace

extern "C" {

int hobi_setup(const double* vertices, int64_t n_v, const int32_t* faces, int64_t n_f, const double* vertex_normals,
               const double* charges, int64_t n_c, double eps1, double eps2, double kappa, const hobi_options* opt,
               hobi_t* out) {
  NvtxRange nvtx_range("hobi_setup");
  return create_handle(vertices, n_v, faces, n_f, vertex_normals, charges, n_c, eps1, eps2, kappa, opt, false, out);
}

int hobi_set_precision(hobi_t h, int32_t precision) {
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (precision != HOBI_FP64 && precision != HOBI_FP32_BULK) return fail(HOBI_ERR_ARG, "unknown precision");
  h->precision = precision;
  return HOBI_OK;
}

int hobi_sizes(hobi_t h, int64_t* n_v, int64_t* n_f, int64_t* n_c, int64_t* n_nodes, int64_t* n_points) {
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (n_points) *n_points = h->nv;
  if (n_v) *n_v = h->nv_mesh;
  if (n_f) *n_f = h->nf;
  if (n_c) *n_c = h->nc;
  if (n_nodes) *n_nodes = h->n_nodes;
  return HOBI_OK;
}

int hobi_matvec(hobi_t h, const double* u, double* Au) {
  NvtxRange nvtx_range("hobi_matvec");
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (!u || !Au) return fail(HOBI_ERR_ARG, "u and Au must be non-NULL");
  if (u == Au) return fail(HOBI_ERR_ARG, "Au must not alias u");
  DeviceGuard guard(h->device);
  const int64_t n = 2 * h->nv;
  HOBI_TRY(h->enter());
  const double* ud = u;
  double* ad = Au;
  if (!h->mem_device) {
    HOBI_CK(cudaMemcpyAsync(h->u_stage, u, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    ud = h->u_stage;
    ad = h->au_stage;
  }
  HOBI_TRY(h->matvec_dev(ud, nullptr, 0, ad));
  if (!h->mem_device) HOBI_CK(cudaMemcpyAsync(Au, ad, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  HOBI_TRY(h->finish());
  HOBI_TRY(h->collect_profile());
  return h->check_farfield();
}

int hobi_rhs(hobi_t h, double* b) {
  if (!h || !b) return fail(HOBI_ERR_ARG, "NULL argument");
  DeviceGuard guard(h->device);
  HOBI_TRY(h->enter());
  HOBI_TRY(h->copy_out(b, h->b, 2 * h->nv));
  return h->finish();
}

}  // extern "C"

namespace {
// GMRES driver. warm: start from x0 (u0, or the handle's current solution when u0 is NULL);
// the residual test stays relative to ||b||.
int solve_impl(hobi_t h, const double* u0, bool warm, double tol, int32_t max_it, double* phi, double* dphi,
               hobi_solve_info* info) {
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (!(tol > 0.0) || max_it < 1) return fail(HOBI_ERR_ARG, "need tol > 0 and max_it >= 1");
  if (warm && !u0 && !h->have_solution)
    return fail(HOBI_ERR_STATE, "no solution to resume from: pass u0 or solve first");
  DeviceGuard guard(h->device);
  const int64_t n = 2 * h->nv;
  const int m = h->restart;
  HOBI_TRY(h->enter());
  HOBI_CK(cudaEventRecord(h->ev_t0, h->stream));
  // ||b|| fixes the relative residual; cold start: x = 0, r = b
  GmresState s0;
  memset(&s0, 0, sizeof s0);
  s0.tol = tol;
  *h->st_host = s0;
  HOBI_CK(cudaMemcpyAsync(h->st, h->st_host, sizeof(GmresState), cudaMemcpyHostToDevice, h->stream));
  if (warm) {
    if (u0) HOBI_TRY(h->copy_in(h->x, u0, n));
  } else {
    HOBI_CK(cudaMemsetAsync(h->x, 0, sizeof(double) * n, h->stream));
  }
  HOBI_CK(cudaMemcpyAsync(h->Vb, h->b, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  HOBI_CK(launch_dots(nullptr, 0, h->Vb, n, h->st, 1, h->dpart, h->stream));
  HOBI_CK(launch_reduce_dots(h->dpart, m, h->st, 1, h->nrm, nullptr, 0, h->stream));
  HOBI_CK(launch_cycle_start(h->Vb, n, h->nrm, h->st, h->g, m, 1, h->stream));
  h->launches += 3;
  if (warm) {  // r0 = b - A x0 replaces the first basis vector
    HOBI_TRY(h->matvec_dev(h->x, nullptr, 0, h->w));
    HOBI_CK(launch_residual_start(h->b, h->w, h->Vb, n, h->stream));
    HOBI_CK(launch_dots(nullptr, 0, h->Vb, n, h->st, 1, h->dpart, h->stream));
    HOBI_CK(launch_reduce_dots(h->dpart, m, h->st, 1, h->nrm, nullptr, 0, h->stream));
    HOBI_CK(launch_cycle_start(h->Vb, n, h->nrm, h->st, h->g, m, 0, h->stream));
    h->launches += 4;
  }
  HOBI_TRY(h->read_state());
  std::vector<double> hist;
  hist.push_back(h->st_host->rel);
  bool done = h->st_host->converged || h->st_host->breakdown;
  while (!done) {
    for (int kk = 0; kk < m; ++kk) {
      if (h->st_host->it >= max_it) break;
      HOBI_TRY(h->run_iteration());
      HOBI_TRY(h->read_state());
      hist.push_back(h->st_host->rel);
      if (h->st_host->converged || h->st_host->breakdown) break;
    }
    HOBI_CK(launch_finish_cycle(h->H, m, h->g, h->st, h->y, h->Vb, n, h->x, n, h->stream));
    h->launches += 2;
    if (h->st_host->converged || h->st_host->breakdown || h->st_host->it >= max_it) break;
    // restart from r = b - A x
    HOBI_TRY(h->matvec_dev(h->x, nullptr, 0, h->w));
    HOBI_CK(launch_residual_start(h->b, h->w, h->Vb, n, h->stream));
    HOBI_CK(launch_dots(nullptr, 0, h->Vb, n, h->st, 1, h->dpart, h->stream));
    HOBI_CK(launch_reduce_dots(h->dpart, m, h->st, 1, h->nrm, nullptr, 0, h->stream));
    HOBI_CK(launch_cycle_start(h->Vb, n, h->nrm, h->st, h->g, m, 0, h->stream));
    h->launches += 4;
    HOBI_TRY(h->read_state());
    done = h->st_host->converged || h->st_host->breakdown;
  }
  HOBI_CK(cudaEventRecord(h->ev_t1, h->stream));
  if (phi) HOBI_TRY(h->copy_out(phi, h->x, h->nv));
  if (dphi) HOBI_TRY(h->copy_out(dphi, h->x + h->nv, h->nv));
  HOBI_TRY(h->finish());
  HOBI_CK(cudaEventSynchronize(h->ev_t1));
  HOBI_TRY(h->collect_profile());
  HOBI_TRY(h->check_farfield());
  h->have_solution = true;
  const GmresState fs = *h->st_host;
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1);
    info->iterations = fs.it;
    info->converged = fs.converged;
    info->rel_residual = fs.rel;
    info->solve_ms = ms;
    const double per_matvec = h->fast_active(h->precision == HOBI_FP32_BULK)
                                  ? (double)(h->fast_direct_pairs + h->fast_approx_pairs)
                                  : (double)h->nv * (double)h->n_nodes;
    info->farfield_pairs = (double)fs.it * per_matvec;
    if (info->resid_history && info->resid_capacity > 0) {
      int cnt = (int)hist.size() < info->resid_capacity ? (int)hist.size() : info->resid_capacity;
      for (int i = 0; i < cnt; ++i) info->resid_history[i] = hist[i];
    }
  }
  if (fs.converged) return HOBI_OK;
  if (fs.breakdown) return fail(HOBI_ERR_BREAKDOWN, "GMRES breakdown (zero or non-finite Arnoldi norm)");
  return fail(HOBI_ERR_NOT_CONVERGED, "GMRES did not reach tol within max_it iterations (rel residual " +
                                          std::to_string(fs.rel) + ")");
}

// Mixed-precision solve (iterative refinement): the correction equation A d = r is solved by
// FP32-bulk GMRES to 1e-6, the residual r = b - A u of the accumulated u is formed with the FP64
// far field, until ||r|| / ||b|| <= tol on the FP64 operator.
int solve_refined_impl(hobi_t h, double tol, int32_t max_refine, int32_t max_it, double* phi, double* dphi,
                       hobi_solve_info* info) {
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (!(tol > 0.0) || max_refine < 1 || max_it < 1)
    return fail(HOBI_ERR_ARG, "need tol > 0, max_refine >= 1 and max_it >= 1");
  DeviceGuard guard(h->device);
  const int64_t n = 2 * h->nv;
  if (!h->ref_x) {
    HOBI_TRY(h->alloc(&h->ref_x, n));
    HOBI_TRY(h->alloc(&h->ref_r, n));
    HOBI_TRY(h->alloc(&h->ref_d, n));
    HOBI_TRY(h->alloc(&h->ref_scal, 1));
    HOBI_CK(cudaEventCreate(&h->ref_t0));
    HOBI_CK(cudaEventCreate(&h->ref_t1));
  }
  HOBI_TRY(h->enter());
  HOBI_CK(cudaEventRecord(h->ref_t0, h->stream));
  auto norm = [&](const double* v, double* out) -> int {
    HOBI_CK(launch_norm2(v, n, h->ref_scal, h->stream));
    HOBI_CK(cudaMemcpyAsync(out, h->ref_scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HOBI_CK(cudaStreamSynchronize(h->stream));
    h->launches += 1;
    return HOBI_OK;
  };
  const int saved = h->precision;
  double bnorm = 0.0, rel = 0.0;
  HOBI_CK(cudaMemsetAsync(h->ref_x, 0, sizeof(double) * n, h->stream));
  HOBI_TRY(norm(h->b, &bnorm));
  std::vector<double> hist;
  int inner_it = 0, status = HOBI_OK;
  double pairs = 0.0;
  for (int k = 0; bnorm > 0.0; ++k) {
    if (k == 0) {
      HOBI_CK(cudaMemcpyAsync(h->ref_r, h->b, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
    } else {  // r = b - A u with the FP64 far field
      h->precision = HOBI_FP64;
      HOBI_TRY(h->matvec_dev(h->ref_x, nullptr, 0, h->w));
      HOBI_CK(launch_residual_start(h->b, h->w, h->ref_r, n, h->stream));
      h->launches += 1;
      pairs += (double)h->nv * (double)h->n_nodes;
    }
    double rnorm = 0.0;
    HOBI_TRY(norm(h->ref_r, &rnorm));
    rel = rnorm / bnorm;
    hist.push_back(rel);
    if (rel <= tol || k >= max_refine) break;
    // FP32-bulk GMRES on A d = r (b and x of the handle point at r and d meanwhile)
    h->precision = HOBI_FP32_BULK;
    std::swap(h->b, h->ref_r);
    std::swap(h->x, h->ref_d);
    hobi_solve_info ii;
    memset(&ii, 0, sizeof ii);
    const int r = solve_impl(h, nullptr, false, 1e-6, max_it, nullptr, nullptr, &ii);
    std::swap(h->b, h->ref_r);
    std::swap(h->x, h->ref_d);
    h->precision = saved;
    inner_it += ii.iterations;
    pairs += ii.farfield_pairs;
    if (r != HOBI_OK && r != HOBI_ERR_NOT_CONVERGED) return r;
    HOBI_CK(launch_add_in_place(h->ref_x, h->ref_d, n, h->stream));
    h->launches += 1;
  }
  h->precision = saved;
  HOBI_CK(cudaMemcpyAsync(h->x, h->ref_x, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  HOBI_CK(cudaEventRecord(h->ref_t1, h->stream));
  if (phi) HOBI_TRY(h->copy_out(phi, h->x, h->nv));
  if (dphi) HOBI_TRY(h->copy_out(dphi, h->x + h->nv, h->nv));
  HOBI_TRY(h->finish());
  HOBI_CK(cudaEventSynchronize(h->ref_t1));
  h->have_solution = true;
  if (rel > tol) status = fail(HOBI_ERR_NOT_CONVERGED, "refinement did not reach tol within max_refine steps "
                                                       "(FP64 rel residual " + std::to_string(rel) + ")");
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ref_t0, h->ref_t1);
    info->iterations = inner_it;
    info->converged = rel <= tol;
    info->rel_residual = rel;
    info->solve_ms = ms;
    info->farfield_pairs = pairs;
    if (info->resid_history && info->resid_capacity > 0) {
      const int cnt = (int)hist.size() < info->resid_capacity ? (int)hist.size() : info->resid_capacity;
      for (int i = 0; i < cnt; ++i) info->resid_history[i] = hist[i];
    }
  }
  return status;
}
}  // namespace

extern "C" {

int hobi_solve(hobi_t h, double tol, int32_t max_it, double* phi, double* dphi, hobi_solve_info* info) {
  NvtxRange nvtx_range("hobi_solve");
  return solve_impl(h, nullptr, false, tol, max_it, phi, dphi, info);
}

int hobi_solve_refined(hobi_t h, double tol, int32_t max_refine, int32_t max_it, double* phi, double* dphi,
                       hobi_solve_info* info) {
  NvtxRange nvtx_range("hobi_solve_refined");
  return solve_refined_impl(h, tol, max_refine, max_it, phi, dphi, info);
}

int hobi_solve_from(hobi_t h, const double* u0, double tol, int32_t max_it, double* phi, double* dphi,
                    hobi_solve_info* info) {
  NvtxRange nvtx_range("hobi_solve_from");
  return solve_impl(h, u0, true, tol, max_it, phi, dphi, info);
}

int hobi_set_solution(hobi_t h, const double* u) {
  if (!h || !u) return fail(HOBI_ERR_ARG, "NULL argument");
  DeviceGuard guard(h->device);
  HOBI_TRY(h->enter());
  HOBI_TRY(h->copy_in(h->x, u, 2 * h->nv));
  HOBI_TRY(h->finish());
  h->have_solution = true;
  return HOBI_OK;
}

int hobi_get_solution(hobi_t h, double* u) {
  if (!h || !u) return fail(HOBI_ERR_ARG, "NULL argument");
  if (!h->have_solution) return fail(HOBI_ERR_STATE, "no solution: call hobi_solve or hobi_set_solution first");
  DeviceGuard guard(h->device);
  HOBI_TRY(h->enter());
  HOBI_TRY(h->copy_out(u, h->x, 2 * h->nv));
  return h->finish();
}

int hobi_reaction_potential(hobi_t h, const double* points, int64_t n_points, double* phi) {
  NvtxRange nvtx_range("hobi_reaction_potential");
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (n_points < 0 || (n_points > 0 && (!points || !phi))) return fail(HOBI_ERR_ARG, "bad points/phi arguments");
  if (!h->have_solution) return fail(HOBI_ERR_STATE, "no solution: call hobi_solve or hobi_set_solution first");
  if (n_points == 0) return HOBI_OK;
  if (n_points > (int64_t(1) << 28)) return fail(HOBI_ERR_ARG, "too many points");
  DeviceGuard guard(h->device);
  HOBI_TRY(h->enter());
  HOBI_TRY(h->ensure_point_buffers(n_points));
  HOBI_TRY(h->copy_in(h->pts_in, points, 3 * n_points));
  HOBI_CK(launch_points((int)n_points, h->pts_in, 3, h->center, h->xs, h->ptgt32, h->ptgt64, h->stream));
  h->launches += 1;
  HOBI_TRY(h->reaction_dev(n_points, h->ptgt32, h->ptgt64, h->phi_pts));
  HOBI_TRY(h->copy_out(phi, h->phi_pts, n_points));
  HOBI_TRY(h->finish());
  HOBI_TRY(h->collect_profile());
  return h->check_farfield();
}

int hobi_energy(hobi_t h, double* e_sol) {
  NvtxRange nvtx_range("hobi_energy");
  if (!h || !e_sol) return fail(HOBI_ERR_ARG, "NULL argument");
  if (!h->have_solution) return fail(HOBI_ERR_STATE, "no solution: call hobi_solve or hobi_set_solution first");
  DeviceGuard guard(h->device);
  if (h->nc == 0) {
    *e_sol = 0.0;
    return HOBI_OK;
  }
  HOBI_TRY(h->enter());
  HOBI_TRY(h->ensure_point_buffers(h->nc));
  HOBI_TRY(h->reaction_dev(h->nc, h->ctgt32, h->ctgt64, h->phi_pts));
  HOBI_CK(launch_energy_sum((int)h->nc, h->Q, h->phi_pts, h->e_dev, h->stream));
  h->launches += 1;
  HOBI_CK(cudaMemcpyAsync(h->host_scalar, h->e_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HOBI_TRY(h->leave());
  HOBI_CK(cudaStreamSynchronize(h->stream));
  HOBI_TRY(h->collect_profile());
  HOBI_TRY(h->check_farfield());
  *e_sol = *h->host_scalar;
  return HOBI_OK;
}

int hobi_get_nodes(hobi_t h, double* y, double* nu, double* W) {
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  DeviceGuard guard(h->device);
  HOBI_TRY(h->enter());
  if (y) HOBI_TRY(h->copy_out(y, h->ny, 3 * h->n_nodes));
  if (nu) HOBI_TRY(h->copy_out(nu, h->nnu, 3 * h->n_nodes));
  if (W) HOBI_TRY(h->copy_out(W, h->nW, 3 * h->n_nodes));
  return h->finish();
}

int hobi_get_correction(hobi_t h, int64_t* n_entries, int32_t* vertex, int32_t* face, double* coeff) {
  if (!h || !n_entries) return fail(HOBI_ERR_ARG, "NULL argument");
  *n_entries = h->scheme == HOBI_SCHEME_LOBI ? 0 : 3 * h->nf;
  if (*n_entries == 0) return HOBI_OK;
  if (!vertex && !face && !coeff) return HOBI_OK;
  DeviceGuard guard(h->device);
  HOBI_TRY(h->enter());
  const size_t ne = (size_t)(3 * h->nf);
  if (vertex) HOBI_CK(cudaMemcpyAsync(vertex, h->entry_vertex, sizeof(int) * ne, cudaMemcpyDeviceToHost, h->stream));
  if (face) HOBI_CK(cudaMemcpyAsync(face, h->inc_face, sizeof(int) * ne, cudaMemcpyDeviceToHost, h->stream));
  if (coeff) HOBI_CK(cudaMemcpyAsync(coeff, h->corr, sizeof(double) * 12 * ne, cudaMemcpyDeviceToHost, h->stream));
  HOBI_TRY(h->leave());
  HOBI_CK(cudaStreamSynchronize(h->stream));
  return HOBI_OK;
}

int hobi_profile_enable(hobi_t h, int32_t on) {
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  h->prof = on != 0;
  return HOBI_OK;
}

int hobi_profile_read(hobi_t h, double* farfield_ms, int64_t* launches, double* pairs) {
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  DeviceGuard guard(h->device);
  HOBI_TRY(h->collect_profile());
  if (farfield_ms) *farfield_ms = h->prof_ms;
  if (launches) *launches = h->prof_launches;
  if (pairs) *pairs = h->prof_pairs;
  h->prof_ms = 0.0;
  h->prof_launches = 0;
  h->prof_pairs = 0.0;
  return HOBI_OK;
}

int hobi_plan_info(hobi_t h, int32_t* shape, int32_t* chunks, int32_t* tuned) {
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (shape) *shape = h->plan[1].shape;
  if (chunks) *chunks = h->plan[1].chunks;
  if (tuned) *tuned = h->tuned;
  return HOBI_OK;
}

int hobi_fast_info(hobi_t h, int64_t* direct_pairs, int64_t* approx_pairs, int32_t* batches, int32_t* proxy_clusters,
                   int32_t* tasks) {
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (direct_pairs) *direct_pairs = h->fast_direct_pairs;
  if (approx_pairs) *approx_pairs = h->fast_approx_pairs;
  if (batches) *batches = h->fast_batches;
  if (proxy_clusters) *proxy_clusters = h->fast_npc;
  if (tasks) *tasks = h->fast_ntasks;
  return HOBI_OK;
}

int hobi_fast_plan_stats(const double* nodes, int64_t n_nodes, const double* targets, int64_t n_targets,
                         int32_t degree, double theta, int64_t* direct_pairs, int64_t* approx_pairs,
                         int32_t* batches, int32_t* proxy_clusters) {
  if (!nodes || !targets || n_nodes < 1 || n_targets < 1) return fail(HOBI_ERR_ARG, "need nodes and targets");
  if (n_nodes > INT32_MAX / 2 || n_targets > INT32_MAX / 2) return fail(HOBI_ERR_ARG, "too many points");
  if (degree < 2 || degree > kFastMaxDegree) return fail(HOBI_ERR_ARG, "degree must be 2..10");
  if (!(theta > 0.0 && theta <= 1.0)) return fail(HOBI_ERR_ARG, "theta must be in (0, 1]");
  FastPlanHost P;
  const double origin[3] = {0.0, 0.0, 0.0};
  build_fast_plan(nodes, (int)n_nodes, targets, (int)n_targets, origin, 1.0, degree, theta, 1, 0, &P);
  if (direct_pairs) *direct_pairs = P.direct_pairs;
  if (approx_pairs) *approx_pairs = P.approx_pairs;
  if (batches) *batches = (int32_t)P.batch.size();
  if (proxy_clusters) *proxy_clusters = (int32_t)P.pc_offset.size();
  return HOBI_OK;
}

int hobi_fp64_pair_functions(const double* x, int64_t n, double* rsqrt_x, double* exp_neg_x) {
  if (n < 0 || n > (int64_t)1 << 24) return fail(HOBI_ERR_ARG, "n must be in [0, 2^24]");
  if (n == 0) return HOBI_OK;
  if (!x || !rsqrt_x || !exp_neg_x) return fail(HOBI_ERR_ARG, "NULL argument");
  for (int64_t k = 0; k < n; ++k)
    if (!(x[k] >= 0.0 && x[k] <= 1e12)) return fail(HOBI_ERR_ARG, "x must be in [0, 1e12]");
  double* d = nullptr;
  const size_t bytes = sizeof(double) * (size_t)n;
  if (cudaMalloc(&d, 3 * bytes) != cudaSuccess) return fail(HOBI_ERR_NOMEM, "cudaMalloc failed");
  cudaError_t e = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_fp64_pair_functions(d, n, d + n, d + 2 * n, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(rsqrt_x, d + n, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(exp_neg_x, d + 2 * n, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(HOBI_ERR_CUDA, std::string("hobi_fp64_pair_functions: ") + cudaGetErrorString(e));
  return HOBI_OK;
}

int hobi_kernel_launches(hobi_t h, int64_t* n) {
  if (!h || !n) return fail(HOBI_ERR_ARG, "NULL argument");
  *n = h->launches;
  return HOBI_OK;
}

void hobi_destroy(hobi_t h) {
  if (!h) return;
  DeviceGuard guard(h->device);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Reaction potential without any device allocation.
//
// For callers that must not allocate device memory once they are running: a host whose device
// memory is owned by another allocator (a framework's caching pool that holds the GPU's free
// memory, so a cudaMalloc from this library would fail or break the pool's accounting), a
// service whose memory footprint is fixed when it starts, and a latency-bound loop that cannot
// pay cudaMalloc's cost and its synchronisation with the other streams of the device. The per-call
// scratch (the caller's points as targets, the per-chunk partial sums and the reduced potentials)
// lives in one file-scope device array of fixed size instead of buffers allocated on demand; the
// handle's own tables were allocated by hobi_setup beforehand.
namespace {

constexpr int64_t kNoAllocMaxPoints = 4096;  // points per call
constexpr int kNoAllocMaxChunks = 64;        // source chunks of the far-field sum
// layout: points [3n] double | targets64 [8n] double | phi [n] double | partials [64 n] double |
//         targets32 [2n] float4
constexpr size_t kNoAllocBytes = (size_t)kNoAllocMaxPoints * (3 + 8 + 1 + kNoAllocMaxChunks) * sizeof(double) +
                                 (size_t)kNoAllocMaxPoints * 2 * sizeof(float4);

}  // namespace

// 2.5 MiB, shared by every call on a device; resident on every GPU that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on `dev` (current device). Looked up once per device:
// in host code the array's name is only a host-side stand-in, not a device address.
int noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(HOBI_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(HOBI_ERR_CUDA, std::string("cudaGetSymbolAddress(no-allocation scratch): ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_addr[dev];
  return HOBI_OK;
}

}  // namespace

extern "C" int hobi_reaction_potential_noalloc(hobi_t h, const double* points, int64_t n_points, double* phi) {
  NvtxRange nvtx_range("hobi_reaction_potential_noalloc");
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (n_points < 0 || (n_points > 0 && (!points || !phi))) return fail(HOBI_ERR_ARG, "bad points/phi arguments");
  if (n_points > kNoAllocMaxPoints)
    return fail(HOBI_ERR_ARG, "n_points = " + std::to_string(n_points) + " exceeds the no-allocation limit of " +
                                  std::to_string(kNoAllocMaxPoints) + " points per call");
  if (!h->have_solution) return fail(HOBI_ERR_STATE, "no solution: call hobi_solve or hobi_set_solution first");
  if (n_points == 0) return HOBI_OK;
  DeviceGuard guard(h->device);
  unsigned char* base = nullptr;
  HOBI_TRY(noalloc_scratch(h->device, &base));
  const int64_t n = n_points;
  double* pts = reinterpret_cast<double*>(base);
  double* t64 = pts + 3 * kNoAllocMaxPoints;
  double* phi_d = t64 + 8 * kNoAllocMaxPoints;
  double* part = phi_d + kNoAllocMaxPoints;
  float4* t32 = reinterpret_cast<float4*>(part + (size_t)kNoAllocMaxChunks * kNoAllocMaxPoints);
  const bool fp32 = h->precision == HOBI_FP32_BULK;
  FarFieldPlan p = plan_farfield(fp32, (int)n, (int)h->n_pad, false, h->num_sms, farfield_blocks_per_sm(fp32, false));
  if (p.chunks > kNoAllocMaxChunks) {
    p.tiles_per_chunk = (p.n_tiles + kNoAllocMaxChunks - 1) / kNoAllocMaxChunks;
    p.chunks = (p.n_tiles + p.tiles_per_chunk - 1) / p.tiles_per_chunk;
  }
  // every (chunk, point) partial is written by the far-field kernel before it is read, so the
  // scratch left over from an earlier call needs no clearing
  HOBI_TRY(h->enter());
  HOBI_TRY(h->copy_in(pts, points, 3 * n));
  HOBI_CK(launch_points((int)n, pts, 3, h->center, h->xs, t32, t64, h->stream));
  HOBI_TRY(h->gather(fp32, h->x, nullptr, 0));
  HOBI_TRY(h->farfield(fp32, p, t32, t64, part));  // timed like every far-field launch when profiling is on
  HOBI_CK(launch_reduce_points((int)n, p.chunks, part, phi_d, h->stream));
  h->launches += 4;
  HOBI_TRY(h->copy_out(phi, phi_d, n));
  HOBI_TRY(h->finish());
  HOBI_TRY(h->collect_profile());
  return h->check_farfield();
}

// =============================================================================================
// Batched solve: many molecules, one far-field launch per GMRES step (one block per task in FP32,
// persistent blocks pulling tasks in FP64).
// =============================================================================================
struct hobi_batch_ctx {
  int device = 0;
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  int mem_device = 0, precision = HOBI_FP32_BULK, restart = 50, use_graph = 1, num_sms = 1;
  double eps = 80, kappa = 0;
  int nmol = 0;
  std::vector<hobi_t> subs;
  std::vector<MolDesc> mols_h;
  int* ff_err = nullptr;  // far-field tile pipeline timeout flag (device)
  std::vector<int64_t> vert_off_h, node_off_h, charge_off_h;
  int64_t N = 0, total_nodes = 0, total_verts = 0;
  std::vector<void*> allocs;
  MolDesc* mols = nullptr;
  FFTask *tasks[2] = {nullptr, nullptr};
  int ntasks[2] = {0, 0};
  int* counter = nullptr;
  int64_t *node_off = nullptr, *vert_off = nullptr;
  Segment* seg = nullptr;
  int nseg = 0;
  int* mol_seg = nullptr;
  double *b = nullptr, *x = nullptr, *w = nullptr, *Vb = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr;
  double *g = nullptr, *y = nullptr, *hcol = nullptr, *cvec = nullptr, *nrm = nullptr, *dpart = nullptr;
  double *u_stage = nullptr, *au_stage = nullptr;
  BatchState* gs = nullptr;
  MolState* ms = nullptr;
  BatchState* gs_host = nullptr;  // pinned
  MolState* ms_host = nullptr;    // pinned
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [precision][profiling]
  bool capturing = false, have_solution = false;
  int64_t launches = 0;
  int ff_grid[2] = {1, 1};
  // fast summation of the FP32 far field for the molecules big enough to gain from it
  int fast_degree = 0, nfup = 0, nfpcs = 0;
  double fast_theta = 0.7;
  FastUpItemB* fup = nullptr;
  FastPCB* fpcs = nullptr;
  std::vector<double> pairs32;  // FP32 pair evaluations per molecule and far-field launch
  // far-field timing (events around each launch; external event nodes inside captured graphs)
  bool prof = false, prof_pending = false;
  cudaEvent_t pev[2] = {nullptr, nullptr};
  double prof_ms = 0.0, prof_pairs = 0.0, pairs_pending = 0.0;
  int64_t prof_launches = 0;
  // pair evaluations of one batched far-field launch over the molecules still iterating
  double active_pairs() const {
    double p = 0.0;
    for (int i = 0; i < nmol; ++i)
      if (!ms_host || (!ms_host[i].converged && !ms_host[i].breakdown)) p += mol_pairs(i);
    return p;
  }
  double mol_pairs(int i) const {
    return precision == HOBI_FP32_BULK ? pairs32[i] : (double)mols_h[i].nv * mols_h[i].n_nodes;
  }
  int prof_collect() {
    if (!prof_pending) return HOBI_OK;
    float ms = 0.f;
    HOBI_CK(cudaEventElapsedTime(&ms, pev[0], pev[1]));
    prof_ms += ms;
    prof_launches += 1;
    prof_pairs += pairs_pending;
    prof_pending = false;
    return HOBI_OK;
  }

  template <class T>
  int alloc(T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(HOBI_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    }
    allocs.push_back(q);
    *p = static_cast<T*>(q);
    return HOBI_OK;
  }
  int enter() {
    HOBI_CK(cudaEventRecord(ev_in, user_stream));
    HOBI_CK(cudaStreamWaitEvent(stream, ev_in, 0));
    return HOBI_OK;
  }
  int leave() {
    HOBI_CK(cudaEventRecord(ev_out, stream));
    HOBI_CK(cudaStreamWaitEvent(user_stream, ev_out, 0));
    return HOBI_OK;
  }
  int ldc() const { return restart + 1; }

  // Au = A u on every molecule (u = base + (*kptr) ld); masked molecules (ms) are skipped
  int matvec(const double* u, const int* kptr, int64_t ld, double* Au, const MolState* mask) {
    const bool fp32 = precision == HOBI_FP32_BULK;
    HOBI_CK(launch_gather_batch(fp32, mols, nmol, node_off, total_nodes, u, kptr, ld, mask, stream));
    if (prof) {
      for (auto& e : pev)
        if (!e) HOBI_CK(cudaEventCreate(&e));
      HOBI_CK(cudaEventRecordWithFlags(pev[0], stream, capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
    }
    if (fp32 && nfup > 0) {  // proxy densities of the molecules that use fast summation
      HOBI_CK(launch_fast_upward_batch(nfup, fup, nfpcs, fpcs, mols, mask, fast_degree, eps, stream));
      if (!capturing) launches += 2;
    }
    HOBI_CK(launch_farfield_batch(fp32, mols, tasks[fp32], ntasks[fp32], counter, mask, eps, kappa, ff_grid[fp32],
                                  ff_err, stream));
    if (prof) {
      HOBI_CK(cudaEventRecordWithFlags(pev[1], stream, capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
      if (!capturing) {
        // timed below once the stream has reached the end event
        pairs_pending = mask ? active_pairs() : active_pairs_all();
        prof_pending = true;
      }
    }
    HOBI_CK(launch_combine_batch(mols, nmol, vert_off, total_verts, u, kptr, ld, Au, mask, fp32, stream));
    if (!capturing) launches += 3;
    return HOBI_OK;
  }

  double active_pairs_all() const {
    double p = 0.0;
    for (int i = 0; i < nmol; ++i) p += mol_pairs(i);
    return p;
  }

  static constexpr int kIterationKernels = 14;
  int iteration() {
    const int m = restart;
    HOBI_TRY(matvec(Vb, &gs->k, N, w, ms));
    for (int pass = 0; pass < 2; ++pass) {
      HOBI_CK(launch_bdots(Vb, N, w, seg, nseg, gs, ms, 0, dpart, stream));
      HOBI_CK(launch_breduce(dpart, nseg, mol_seg, nmol, m, gs, ms, 0, ldc(), cvec, hcol, pass, stream));
      HOBI_CK(launch_baxpy(Vb, N, cvec, ldc(), seg, nseg, gs, ms, w, stream));
    }
    HOBI_CK(launch_bdots(nullptr, 0, w, seg, nseg, gs, ms, 1, dpart, stream));
    HOBI_CK(launch_breduce(dpart, nseg, mol_seg, nmol, m, gs, ms, 1, ldc(), nrm, nullptr, 0, stream));
    HOBI_CK(launch_bgivens(gs, ms, nmol, m, H, cs, sn, g, hcol, nrm, ldc(), stream));
    HOBI_CK(launch_bnext(Vb, N, w, seg, nseg, gs, ms, stream));
    HOBI_CK(launch_badvance(gs, stream));
    if (!capturing) launches += kIterationKernels - 3;
    return HOBI_OK;
  }
  int run_iteration() {
    const int pi = precision == HOBI_FP32_BULK;
    if (!use_graph) return iteration();
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
    if (prof) {
      pairs_pending = active_pairs();  // molecules active when this replay starts
      prof_pending = true;
    }
    HOBI_CK(cudaGraphLaunch(gx, stream));
    launches += kIterationKernels + (pi && nfup > 0 ? 2 : 0);
    return HOBI_OK;
  }
  int read_state() {
    HOBI_CK(cudaMemcpyAsync(gs_host, gs, sizeof(BatchState), cudaMemcpyDeviceToHost, stream));
    HOBI_CK(cudaStreamSynchronize(stream));
    HOBI_TRY(prof_collect());
    HOBI_CK(cudaMemcpyAsync(ms_host, ms, sizeof(MolState) * nmol, cudaMemcpyDeviceToHost, stream));
    HOBI_CK(cudaStreamSynchronize(stream));
    return HOBI_OK;
  }
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
  bool all_done() const {
    for (int i = 0; i < nmol; ++i)
      if (!ms_host[i].converged && !ms_host[i].breakdown) return false;
    return true;
  }
  int start_cycle(int first) {
    HOBI_CK(launch_bdots(nullptr, 0, Vb, seg, nseg, gs, ms, 1, dpart, stream));
    HOBI_CK(launch_breduce(dpart, nseg, mol_seg, nmol, restart, gs, ms, 1, ldc(), nrm, nullptr, 0, stream));
    HOBI_CK(launch_bcycle_start(Vb, seg, nseg, gs, ms, nmol, nrm, ldc(), g, restart, first, stream));
    launches += 4;
    return HOBI_OK;
  }

  ~hobi_batch_ctx() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto& row : graph)
      for (auto& gx : row)
        if (gx) cudaGraphExecDestroy(gx);
    for (cudaEvent_t e : pev)
      if (e) cudaEventDestroy(e);
    for (void* p : allocs)
      if (p) cudaFree(p);
    for (hobi_t s : subs)
      if (s) delete s;
    if (gs_host) cudaFreeHost(gs_host);
    if (ms_host) cudaFreeHost(ms_host);
    for (cudaEvent_t e : {ev_in, ev_out, ev_t0, ev_t1})
      if (e) cudaEventDestroy(e);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

int batch_setup_impl(hobi_batch_ctx* B, const double* vertices, const int64_t* v_off, const int32_t* faces,
                     const int64_t* f_off, const double* normals, const double* charges, const int64_t* c_off,
                     double eps1, double eps2, const hobi_options& o) {
  const int nmol = B->nmol;
  // one single-molecule handle per molecule: validation, nodes, correction table, RHS
  hobi_options so = o;
  so.restart = 1;      // the batch owns the Krylov workspace
  so.use_graph = 0;
  so.fast_degree = 0;  // the batch decides per molecule and builds the plans below
  for (int m = 0; m < nmol; ++m) {
    const int64_t nv = v_off[m + 1] - v_off[m], nf = f_off[m + 1] - f_off[m], nc = c_off[m + 1] - c_off[m];
    hobi_t h = nullptr;
    int r = create_handle(vertices + 3 * v_off[m], nv, faces + 3 * f_off[m], nf, normals + 3 * v_off[m],
                          nc > 0 ? charges + 4 * c_off[m] : nullptr, nc, eps1, eps2, B->kappa, &so, true, &h);
    if (r != HOBI_OK) return fail(r, "molecule " + std::to_string(m) + ": " + g_err);
    B->subs.push_back(h);
  }
  // descriptors, partial-sum buffers and the far-field task lists (one per precision)
  B->vert_off_h.assign(nmol + 1, 0);
  B->node_off_h.assign(nmol + 1, 0);
  std::vector<FFTask> tl[2];
  std::vector<int64_t> cost[2];  // source entries per task (all tasks have the same target count)
  std::vector<FastUpItemB> fup_h;
  std::vector<FastPCB> fpcs_h;
  for (int m = 0; m < nmol; ++m) {
    hobi_ctx* h = B->subs[m];
    MolDesc d;
    d.F = h->F; d.ny = h->ny; d.nnu = h->nnu; d.nW = h->nW; d.center = h->center;
    d.inc_ptr = h->inc_ptr; d.inc_face = h->inc_face; d.corr = h->corr;
    d.tgt32 = h->tgt32; d.tgt64 = h->tgt64; d.src32 = h->src32; d.src64 = h->src64;
    d.nv = (int)h->nv; d.n_nodes = (int)h->n_nodes; d.eps = h->eps; d.xs = h->xs;
    d.u_off = B->N;
    const int n_tiles = (int)(h->n_pad / kTile);
    d.chunks = (n_tiles + kTilesPerTask - 1) / kTilesPerTask;
    d.fast = 0;
    d.fchunks = 0;
    d.fpos = nullptr; d.fsrc = nullptr; d.ftgt = nullptr; d.ftmap = nullptr; d.fseg = nullptr; d.fbatch = nullptr;
    d.faxes = nullptr; d.fhalf = nullptr; d.fpartial = nullptr; d.fpcitems = nullptr; d.fpcoff = nullptr;
    double pairs = (double)h->nv * h->n_nodes;
    if (B->fast_degree > 0 && h->nv >= kFastMinTargets) {
      h->fast_degree = B->fast_degree;
      h->fast_theta = B->fast_theta;
      HOBI_TRY(h->setup_fast(kFastPieceSources));
      const double fp = (double)(h->fast_direct_pairs + h->fast_approx_pairs);
      if (fp <= kFastMaxFraction * pairs) {  // worth it: use the treecode for this molecule
        d.fast = 1;
        d.fchunks = h->fast_chunks;
        d.fpos = h->fast_pos; d.fsrc = h->fast_src; d.ftgt = h->fast_tgt; d.ftmap = h->fast_tmap;
        d.fseg = h->fast_seg; d.fbatch = h->fast_batch; d.faxes = h->fast_axes; d.fhalf = h->fast_half;
        d.fpartial = h->fast_partial; d.fpcitems = h->fast_pcitems; d.fpcoff = h->fast_pcoff;
        pairs = fp;
        for (size_t i = 0; i < h->fast_up_h.size(); ++i) {
          const FastUpItem& it = h->fast_up_h[i];
          fup_h.push_back({m, it.pc, it.n0, it.n1, (int)i});
        }
        for (int pc = 0; pc < h->fast_npc; ++pc) fpcs_h.push_back({m, pc});
      } else {
        h->fast_degree = 0;
      }
    }
    B->pairs32.push_back(pairs);
    HOBI_TRY(B->alloc(&d.part, (size_t)std::max(d.chunks, d.fchunks) * 2 * h->nv));
    for (int fp32 = 0; fp32 < 2; ++fp32) {
      if (fp32 && d.fast) {
        for (size_t q = 0; q < h->fast_tasks_h.size(); ++q) {
          const FastTask& t = h->fast_tasks_h[q];
          tl[fp32].push_back({m, t.batch, t.s0, t.s1, t.chunk, 1});
          cost[fp32].push_back(h->fast_task_cost_h[q]);
        }
        continue;
      }
      const int per_block = fp32 ? kBatchFF32Threads * kFF32Targets : kFF64Threads * kFF64Targets;
      const int tiles = fp32 ? (int)(h->n_pad / kBatchFF32Tile) : n_tiles;
      const int tpt = fp32 ? kBatchFF32TilesPerTask : kTilesPerTask;
      const int tile_nodes = fp32 ? kBatchFF32Tile : kTile;
      const int tt = (int)((h->nv + per_block - 1) / per_block);
      for (int bx = 0; bx < tt; ++bx)
        for (int c = 0; c < d.chunks; ++c) {
          const int t0 = c * tpt, t1 = std::min(tiles, (c + 1) * tpt);
          tl[fp32].push_back({m, bx, t0, t1, c, 0});
          cost[fp32].push_back((int64_t)(t1 - t0) * tile_nodes);
        }
    }
    B->mols_h.push_back(d);
    B->N += 2 * h->nv;
    B->vert_off_h[m + 1] = B->vert_off_h[m] + h->nv;
    B->node_off_h[m + 1] = B->node_off_h[m] + h->n_nodes;
  }
  B->total_verts = B->vert_off_h[nmol];
  B->total_nodes = B->node_off_h[nmol];
  B->nfup = (int)fup_h.size();
  B->nfpcs = (int)fpcs_h.size();
  if (B->nfup > 0) {
    HOBI_TRY(B->alloc(&B->fup, fup_h.size()));
    HOBI_TRY(B->alloc(&B->fpcs, fpcs_h.size()));
    HOBI_CK(cudaMemcpyAsync(B->fup, fup_h.data(), sizeof(FastUpItemB) * fup_h.size(), cudaMemcpyHostToDevice,
                            B->stream));
    HOBI_CK(cudaMemcpyAsync(B->fpcs, fpcs_h.data(), sizeof(FastPCB) * fpcs_h.size(), cudaMemcpyHostToDevice,
                            B->stream));
  }
  for (int fp32 = 0; fp32 < 2; ++fp32) {
    // longest tasks first, so the tail of the dynamic schedule is made of short ones
    std::vector<int> ord(tl[fp32].size());
    for (size_t q = 0; q < ord.size(); ++q) ord[q] = (int)q;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[fp32][a] > cost[fp32][b]; });
    std::vector<FFTask> sorted;
    for (int q : ord) sorted.push_back(tl[fp32][q]);
    tl[fp32].swap(sorted);
    B->ntasks[fp32] = (int)tl[fp32].size();
    HOBI_TRY(B->alloc(&B->tasks[fp32], tl[fp32].size()));
    HOBI_CK(cudaMemcpyAsync(B->tasks[fp32], tl[fp32].data(), sizeof(FFTask) * tl[fp32].size(), cudaMemcpyHostToDevice,
                            B->stream));
    B->ff_grid[fp32] = B->num_sms * farfield_batch_blocks_per_sm(fp32, B->kappa);
  }
  // segments of the concatenated vector
  std::vector<Segment> segs;
  std::vector<int> mol_seg(nmol + 1, 0);
  for (int m = 0; m < nmol; ++m) {
    mol_seg[m] = (int)segs.size();
    const int64_t len = 2 * (int64_t)B->mols_h[m].nv;
    for (int64_t s0 = 0; s0 < len; s0 += kSegLen)
      segs.push_back({B->mols_h[m].u_off + s0, (int)std::min<int64_t>(kSegLen, len - s0), m});
  }
  mol_seg[nmol] = (int)segs.size();
  B->nseg = (int)segs.size();
  HOBI_TRY(B->alloc(&B->mols, nmol));
  HOBI_TRY(B->alloc(&B->seg, segs.size()));
  HOBI_TRY(B->alloc(&B->mol_seg, nmol + 1));
  HOBI_TRY(B->alloc(&B->node_off, nmol + 1));
  HOBI_TRY(B->alloc(&B->vert_off, nmol + 1));
  HOBI_TRY(B->alloc(&B->counter, 1));
  HOBI_TRY(B->alloc(&B->ff_err, 1));
  HOBI_CK(cudaMemsetAsync(B->ff_err, 0, sizeof(int), B->stream));
  HOBI_CK(cudaMemcpyAsync(B->mols, B->mols_h.data(), sizeof(MolDesc) * nmol, cudaMemcpyHostToDevice, B->stream));
  HOBI_CK(cudaMemcpyAsync(B->seg, segs.data(), sizeof(Segment) * segs.size(), cudaMemcpyHostToDevice, B->stream));
  HOBI_CK(cudaMemcpyAsync(B->mol_seg, mol_seg.data(), sizeof(int) * (nmol + 1), cudaMemcpyHostToDevice, B->stream));
  HOBI_CK(cudaMemcpyAsync(B->node_off, B->node_off_h.data(), sizeof(int64_t) * (nmol + 1), cudaMemcpyHostToDevice,
                          B->stream));
  HOBI_CK(cudaMemcpyAsync(B->vert_off, B->vert_off_h.data(), sizeof(int64_t) * (nmol + 1), cudaMemcpyHostToDevice,
                          B->stream));
  // concatenated vectors and the batched Krylov workspace
  const int m = B->restart;
  HOBI_TRY(B->alloc(&B->b, B->N));
  HOBI_TRY(B->alloc(&B->x, B->N));
  HOBI_TRY(B->alloc(&B->w, B->N));
  HOBI_TRY(B->alloc(&B->u_stage, B->N));
  HOBI_TRY(B->alloc(&B->au_stage, B->N));
  HOBI_TRY(B->alloc(&B->Vb, (size_t)(m + 1) * B->N));
  HOBI_TRY(B->alloc(&B->H, (size_t)nmol * (m + 1) * m));
  HOBI_TRY(B->alloc(&B->cs, (size_t)nmol * m));
  HOBI_TRY(B->alloc(&B->sn, (size_t)nmol * m));
  HOBI_TRY(B->alloc(&B->g, (size_t)nmol * (m + 1)));
  HOBI_TRY(B->alloc(&B->y, (size_t)nmol * m));
  HOBI_TRY(B->alloc(&B->hcol, (size_t)nmol * (m + 1)));
  HOBI_TRY(B->alloc(&B->cvec, (size_t)nmol * (m + 1)));
  HOBI_TRY(B->alloc(&B->nrm, (size_t)nmol * (m + 1)));
  HOBI_TRY(B->alloc(&B->dpart, (size_t)(m + 1) * B->nseg));
  HOBI_TRY(B->alloc(&B->gs, 1));
  HOBI_TRY(B->alloc(&B->ms, nmol));
  HOBI_CK(cudaMallocHost(&B->gs_host, sizeof(BatchState)));
  HOBI_CK(cudaMallocHost(&B->ms_host, sizeof(MolState) * nmol));
  for (int i = 0; i < nmol; ++i)
    HOBI_CK(cudaMemcpyAsync(B->b + B->mols_h[i].u_off, B->subs[i]->b, sizeof(double) * 2 * B->mols_h[i].nv,
                            cudaMemcpyDeviceToDevice, B->stream));
  HOBI_CK(cudaStreamSynchronize(B->stream));
  return HOBI_OK;
}

}  // namespace

extern "C" {

int hobi_setup_batch(int32_t n_mol, const double* vertices, const int64_t* vertex_offsets, const int32_t* faces,
                     const int64_t* face_offsets, const double* vertex_normals, const double* charges,
                     const int64_t* charge_offsets, double eps1, double eps2, double kappa, const hobi_options* opt,
                     hobi_batch_t* out) {
  NvtxRange nvtx_range("hobi_setup_batch");
  g_err.clear();
  if (!out) return fail(HOBI_ERR_ARG, "out handle pointer is NULL");
  *out = nullptr;
  if (n_mol < 1) return fail(HOBI_ERR_ARG, "n_mol must be >= 1");
  if (!vertex_offsets || !face_offsets || !charge_offsets || !vertices || !faces || !vertex_normals)
    return fail(HOBI_ERR_ARG, "arrays and offsets must be non-NULL");
  for (int m = 0; m < n_mol; ++m)
    if (vertex_offsets[m + 1] < vertex_offsets[m] || face_offsets[m + 1] < face_offsets[m] ||
        charge_offsets[m + 1] < charge_offsets[m])
      return fail(HOBI_ERR_ARG, "offsets must be non-decreasing");
  if (vertex_offsets[0] != 0 || face_offsets[0] != 0 || charge_offsets[0] != 0)
    return fail(HOBI_ERR_ARG, "offsets must start at 0");
  if (charge_offsets[n_mol] > 0 && !charges) return fail(HOBI_ERR_ARG, "charges is NULL");
  if (!(eps1 > 0.0) || !(eps2 > 0.0) || !(kappa >= 0.0) || !isfinite(eps1) || !isfinite(eps2) || !isfinite(kappa))
    return fail(HOBI_ERR_ARG, "need eps1, eps2 > 0 and kappa >= 0, all finite");
  hobi_options o;
  hobi_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != HOBI_FP64 && o.precision != HOBI_FP32_BULK) return fail(HOBI_ERR_ARG, "unknown precision");
  if (o.scheme != HOBI_SCHEME_HOBI) return fail(HOBI_ERR_ARG, "the batch API supports the HOBI scheme only");
  if (o.fast_degree != 0 && (o.fast_degree < 2 || o.fast_degree > kFastMaxDegree))
    return fail(HOBI_ERR_ARG, "fast_degree must be 0 (direct far field) or 2..10");
  if (o.fast_degree != 0 && !(o.fast_theta > 0.0 && o.fast_theta <= 1.0))
    return fail(HOBI_ERR_ARG, "fast_theta must be in (0, 1]");
  if (o.restart <= 0) o.restart = 50;
  if (o.restart > 200) return fail(HOBI_ERR_ARG, "restart must be <= 200");
  int dev = o.device;
  if (dev < 0) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HOBI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  o.device = dev;
  DeviceGuard guard(dev);
  hobi_batch_ctx* B = new hobi_batch_ctx();
  B->device = dev;
  B->user_stream = static_cast<cudaStream_t>(o.stream);
  B->mem_device = o.mem_device ? 1 : 0;
  B->precision = o.precision;
  B->restart = o.restart;
  B->use_graph = o.use_graph ? 1 : 0;
  B->nmol = n_mol;
  B->eps = eps2 / eps1;
  B->kappa = kappa;
  B->fast_degree = o.fast_degree;
  B->fast_theta = o.fast_theta;
  int r = HOBI_OK;
  do {
    cudaError_t e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&B->ev_t0);
    if (e == cudaSuccess) e = cudaEventCreate(&B->ev_t1);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      r = fail(HOBI_ERR_CUDA, std::string("stream/event setup: ") + cudaGetErrorString(e));
      break;
    }
    r = B->enter();
    if (r != HOBI_OK) break;
    r = batch_setup_impl(B, vertices, vertex_offsets, faces, face_offsets, vertex_normals, charges, charge_offsets, eps1,
                         eps2, o);
    if (r != HOBI_OK) break;
    r = B->leave();
  } while (0);
  if (r != HOBI_OK) {
    std::string msg = g_err;
    delete B;
    g_err = msg;
    return r;
  }
  *out = B;
  return HOBI_OK;
}

int hobi_batch_sizes(hobi_batch_t B, int32_t* n_mol, int64_t* total_vertices, int64_t* total_nodes) {
  if (!B) return fail(HOBI_ERR_ARG, "NULL handle");
  if (n_mol) *n_mol = B->nmol;
  if (total_vertices) *total_vertices = B->total_verts;
  if (total_nodes) *total_nodes = B->total_nodes;
  return HOBI_OK;
}

int hobi_batch_set_precision(hobi_batch_t B, int32_t precision) {
  if (!B) return fail(HOBI_ERR_ARG, "NULL handle");
  if (precision != HOBI_FP64 && precision != HOBI_FP32_BULK) return fail(HOBI_ERR_ARG, "unknown precision");
  B->precision = precision;
  return HOBI_OK;
}

int hobi_matvec_batch(hobi_batch_t B, const double* u, double* Au) {
  NvtxRange nvtx_range("hobi_matvec_batch");
  if (!B || !u || !Au) return fail(HOBI_ERR_ARG, "NULL argument");
  if (u == Au) return fail(HOBI_ERR_ARG, "Au must not alias u");
  DeviceGuard guard(B->device);
  HOBI_TRY(B->enter());
  const double* ud = u;
  double* ad = Au;
  if (!B->mem_device) {
    HOBI_CK(cudaMemcpyAsync(B->u_stage, u, sizeof(double) * B->N, cudaMemcpyHostToDevice, B->stream));
    ud = B->u_stage;
    ad = B->au_stage;
  }
  HOBI_TRY(B->matvec(ud, nullptr, 0, ad, nullptr));
  if (!B->mem_device) HOBI_CK(cudaMemcpyAsync(Au, ad, sizeof(double) * B->N, cudaMemcpyDeviceToHost, B->stream));
  HOBI_TRY(B->leave());
  HOBI_CK(cudaStreamSynchronize(B->stream));
  HOBI_TRY(B->prof_collect());
  return B->check_farfield();
}

int hobi_solve_batch(hobi_batch_t B, double tol, int32_t max_it, double* phi, double* dphi, int32_t* iterations,
                     int32_t* status, hobi_solve_info* info) {
  NvtxRange nvtx_range("hobi_solve_batch");
  if (!B) return fail(HOBI_ERR_ARG, "NULL handle");
  if (!(tol > 0.0) || max_it < 1) return fail(HOBI_ERR_ARG, "need tol > 0 and max_it >= 1");
  DeviceGuard guard(B->device);
  const int nmol = B->nmol, m = B->restart;
  HOBI_TRY(B->enter());
  HOBI_CK(cudaEventRecord(B->ev_t0, B->stream));
  BatchState g0{0, 0};
  *B->gs_host = g0;
  for (int i = 0; i < nmol; ++i) {
    MolState s0;
    memset(&s0, 0, sizeof s0);
    s0.tol = tol;
    B->ms_host[i] = s0;
  }
  HOBI_CK(cudaMemcpyAsync(B->gs, B->gs_host, sizeof(BatchState), cudaMemcpyHostToDevice, B->stream));
  HOBI_CK(cudaMemcpyAsync(B->ms, B->ms_host, sizeof(MolState) * nmol, cudaMemcpyHostToDevice, B->stream));
  HOBI_CK(cudaMemsetAsync(B->x, 0, sizeof(double) * B->N, B->stream));
  HOBI_CK(cudaMemcpyAsync(B->Vb, B->b, sizeof(double) * B->N, cudaMemcpyDeviceToDevice, B->stream));
  HOBI_TRY(B->start_cycle(1));
  HOBI_TRY(B->read_state());
  int it = 0;
  bool done = B->all_done();
  while (!done) {
    for (int kk = 0; kk < m; ++kk) {
      if (it >= max_it) break;
      HOBI_TRY(B->run_iteration());
      ++it;
      HOBI_TRY(B->read_state());
      if (B->all_done()) break;
    }
    HOBI_CK(launch_bfinish(B->H, m, B->g, B->ms, nmol, B->y, B->Vb, B->N, B->seg, B->nseg, B->x, B->stream));
    B->launches += 2;
    if (B->all_done() || it >= max_it) break;
    // restart the unconverged molecules from r = b - A x
    HOBI_TRY(B->matvec(B->x, nullptr, 0, B->w, B->ms));
    HOBI_CK(launch_bresidual(B->b, B->w, B->Vb, B->seg, B->nseg, B->ms, B->stream));
    B->launches += 1;
    HOBI_TRY(B->start_cycle(0));
    HOBI_TRY(B->read_state());
    done = B->all_done();
  }
  HOBI_CK(cudaEventRecord(B->ev_t1, B->stream));
  const cudaMemcpyKind kind = B->mem_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int i = 0; i < nmol; ++i) {
    const MolDesc& d = B->mols_h[i];
    if (phi) HOBI_CK(cudaMemcpyAsync(phi + B->vert_off_h[i], B->x + d.u_off, sizeof(double) * d.nv, kind, B->stream));
    if (dphi)
      HOBI_CK(cudaMemcpyAsync(dphi + B->vert_off_h[i], B->x + d.u_off + d.nv, sizeof(double) * d.nv, kind, B->stream));
  }
  HOBI_TRY(B->leave());
  HOBI_CK(cudaStreamSynchronize(B->stream));
  HOBI_TRY(B->check_farfield());
  B->have_solution = true;
  int n_conv = 0, n_break = 0;
  double worst = 0.0;
  for (int i = 0; i < nmol; ++i) {
    const MolState& s = B->ms_host[i];
    if (iterations) iterations[i] = s.it;
    if (status) status[i] = s.converged ? HOBI_OK : (s.breakdown ? HOBI_ERR_BREAKDOWN : HOBI_ERR_NOT_CONVERGED);
    n_conv += s.converged;
    n_break += s.breakdown && !s.converged;
    worst = std::max(worst, s.rel);
  }
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, B->ev_t0, B->ev_t1);
    info->iterations = it;
    info->converged = n_conv == nmol;
    info->rel_residual = worst;
    info->solve_ms = ms;
    double pairs = 0.0;
    for (int i = 0; i < nmol; ++i) pairs += (double)B->ms_host[i].it * B->mols_h[i].nv * (double)B->mols_h[i].n_nodes;
    info->farfield_pairs = pairs;
  }
  if (n_conv == nmol) return HOBI_OK;
  if (n_break) return fail(HOBI_ERR_BREAKDOWN, std::to_string(n_break) + " molecule(s) broke down");
  return fail(HOBI_ERR_NOT_CONVERGED,
              std::to_string(nmol - n_conv) + " molecule(s) did not reach tol within max_it iterations");
}

int hobi_energy_batch(hobi_batch_t B, double* e_sol) {
  NvtxRange nvtx_range("hobi_energy_batch");
  if (!B || !e_sol) return fail(HOBI_ERR_ARG, "NULL argument");
  if (!B->have_solution) return fail(HOBI_ERR_STATE, "no solution: call hobi_solve_batch first");
  DeviceGuard guard(B->device);
  for (int i = 0; i < B->nmol; ++i) {
    hobi_t h = B->subs[i];
    h->precision = B->precision;
    HOBI_CK(cudaMemcpyAsync(h->x, B->x + B->mols_h[i].u_off, sizeof(double) * 2 * h->nv, cudaMemcpyDeviceToDevice,
                            B->stream));
  }
  HOBI_CK(cudaStreamSynchronize(B->stream));
  for (int i = 0; i < B->nmol; ++i) {
    hobi_t h = B->subs[i];
    h->have_solution = true;
    HOBI_TRY(hobi_energy(h, &e_sol[i]));
    B->launches += h->nc > 0 ? 4 : 0;
  }
  return HOBI_OK;
}

int hobi_batch_profile_enable(hobi_batch_t B, int32_t on) {
  if (!B) return fail(HOBI_ERR_ARG, "NULL handle");
  B->prof = on != 0;
  return HOBI_OK;
}

int hobi_batch_profile_read(hobi_batch_t B, double* farfield_ms, int64_t* launches, double* pairs) {
  if (!B) return fail(HOBI_ERR_ARG, "NULL handle");
  if (farfield_ms) *farfield_ms = B->prof_ms;
  if (launches) *launches = B->prof_launches;
  if (pairs) *pairs = B->prof_pairs;
  B->prof_ms = 0.0;
  B->prof_launches = 0;
  B->prof_pairs = 0.0;
  return HOBI_OK;
}

int hobi_batch_kernel_launches(hobi_batch_t B, int64_t* n) {
  if (!B || !n) return fail(HOBI_ERR_ARG, "NULL argument");
  int64_t s = B->launches;
  for (hobi_t h : B->subs) s += h->launches;
  *n = s;
  return HOBI_OK;
}

void hobi_destroy_batch(hobi_batch_t B) {
  if (!B) return;
  DeviceGuard guard(B->device);
  delete B;
}

}  // extern "C"
