// hobi_batch.cu -- the batched C ABI of include/hobi.h (hobi_*_batch): many molecules with the
// same eps1, eps2, kappa solved together. Each molecule's tables come from a single-molecule
// handle (hobi_host.cuh); the batch owns the concatenated Krylov workspace, the far-field task
// lists and the captured GMRES iteration.
#include <atomic>
#include <thread>

#include "hobi_host.cuh"

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
  DeviceArena arena;  // the batch's buffers and its member handles' tables
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
  int gmres_scaling = 1;      // GMRES on the D^-1-scaled unknowns of each molecule
  double* dscale = nullptr;   // [N] scale factor per unknown (gmres_scaling)
  double* zvec = nullptr;     // [N] D^-1 times the current Arnoldi vector
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
    cudaError_t e = arena.get(&q, bytes, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(HOBI_ERR_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                      cudaGetErrorString(e));
    }
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
    if (gmres_scaling) {  // w = A D^-1 v_k on every active molecule
      HOBI_CK(launch_scale_column(Vb, N, &gs->k, dscale, zvec, N, stream));
      if (!capturing) launches += 1;
      HOBI_TRY(matvec(zvec, nullptr, 0, w, ms));
    } else {
      HOBI_TRY(matvec(Vb, &gs->k, N, w, ms));
    }
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
    launches += kIterationKernels + (pi && nfup > 0 ? 2 : 0) + (gmres_scaling ? 1 : 0);
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
    for (hobi_t s : subs)
      if (s) delete s;
    arena.release_all(stream);  // after the members: their last work is ordered before this
    if (gs_host) cudaFreeHost(gs_host);
    if (ms_host) cudaFreeHost(ms_host);
    for (cudaEvent_t e : {ev_in, ev_out, ev_t0, ev_t1})
      if (e) cudaEventDestroy(e);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

constexpr int kSetupThreads = 8;  // host threads that build a batch's member handles

int batch_setup_impl(hobi_batch_ctx* B, const double* vertices, const int64_t* v_off, const int32_t* faces,
                     const int64_t* f_off, const double* normals, const double* charges, const int64_t* c_off,
                     double eps1, double eps2, const hobi_options& o) {
  const int nmol = B->nmol;
  // one single-molecule handle per molecule: validation, nodes, correction table, RHS
  hobi_options so = o;
  so.restart = 1;      // the batch owns the Krylov workspace
  so.use_graph = 0;
  so.fast_degree = 0;  // the batch decides per molecule and builds the plans below
  so.gmres_scaling = 0;
  // The members are independent: host threads build them concurrently, each on its own stream,
  // so their small kernels and host round trips overlap. Every handle made is kept (the batch's
  // destructor frees them); the first failing molecule in index order is reported.
  std::vector<hobi_t> made(nmol, nullptr);
  std::vector<int> rc(nmol, HOBI_OK);
  std::vector<std::string> msg(nmol);
  std::atomic<int> next{0};
  auto build = [&]() {
    for (int m = next.fetch_add(1); m < nmol; m = next.fetch_add(1)) {
      const int64_t nv = v_off[m + 1] - v_off[m], nf = f_off[m + 1] - f_off[m], nc = c_off[m + 1] - c_off[m];
      rc[m] = host_guard([&] {
        const int r = create_handle(vertices + 3 * v_off[m], nv, faces + 3 * f_off[m], nf, normals + 3 * v_off[m],
                                    nc > 0 ? charges + 4 * c_off[m] : nullptr, nc, eps1, eps2, B->kappa, &so, true,
                                    &made[m], &B->arena);
        if (r != HOBI_OK) msg[m] = g_err;
        return r;
      });
      if (rc[m] != HOBI_OK && msg[m].empty()) msg[m] = g_err;
    }
  };
  const int nthreads = std::min(nmol, kSetupThreads);
  std::vector<std::thread> workers;
  for (int t = 1; t < nthreads; ++t) {
    try {
      workers.emplace_back(build);
    } catch (...) {  // no thread to be had: the threads that exist take the remaining molecules
      break;
    }
  }
  build();
  for (auto& t : workers) t.join();
  B->subs = made;
  for (int m = 0; m < nmol; ++m)
    if (rc[m] != HOBI_OK) return fail(rc[m], "molecule " + std::to_string(m) + ": " + msg[m]);
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
  if (B->gmres_scaling) {  // per molecule: 1/((1+eps)/2) on the first n_v unknowns, 1/((1+1/eps)/2) on the rest
    HOBI_TRY(B->alloc(&B->dscale, B->N));
    HOBI_TRY(B->alloc(&B->zvec, B->N));
    for (int i = 0; i < nmol; ++i)
      HOBI_CK(launch_fill_scale(B->dscale + B->mols_h[i].u_off, B->mols_h[i].nv, 1.0 / (0.5 * (1.0 + B->eps)),
                                1.0 / (0.5 * (1.0 + 1.0 / B->eps)), B->stream));
    B->launches += nmol;
  }
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
  if (o.gmres_scaling != 0 && o.gmres_scaling != 1) return fail(HOBI_ERR_ARG, "gmres_scaling must be 0 or 1");
  int dev = o.device;
  if (dev < 0) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HOBI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  o.device = dev;
  DeviceGuard guard(dev);
  hobi_batch_ctx* B = new (std::nothrow) hobi_batch_ctx();
  if (!B) return fail(HOBI_ERR_NOMEM, "host allocation of the batch handle failed");
  B->device = dev;
  B->arena.device = dev;
  B->arena.chunk = size_t(32) << 20;  // one arena for all members: larger blocks
  B->arena.direct = size_t(8) << 20;
  B->arena.shared = true;
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
  B->gmres_scaling = o.gmres_scaling;
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
    B->arena.home = B->stream;
    r = B->enter();
    if (r != HOBI_OK) break;
    r = host_guard([&] {
      return batch_setup_impl(B, vertices, vertex_offsets, faces, face_offsets, vertex_normals, charges,
                              charge_offsets, eps1, eps2, o);
    });
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
    HOBI_CK(launch_bfinish(B->H, m, B->g, B->ms, nmol, B->y, B->Vb, B->N, B->seg, B->nseg, B->x, B->dscale,
                              B->stream));
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
  // queue every member's energy on its own stream, then wait for each
  for (int i = 0; i < B->nmol; ++i) {
    hobi_t h = B->subs[i];
    h->have_solution = true;
    HOBI_TRY(energy_enqueue(h));
  }
  for (int i = 0; i < B->nmol; ++i) HOBI_TRY(energy_finish(B->subs[i], &e_sol[i]));
  return HOBI_OK;
}

int hobi_reaction_forces_batch(hobi_batch_t B, double* forces) {
  NvtxRange nvtx_range("hobi_reaction_forces_batch");
  if (!B) return fail(HOBI_ERR_ARG, "NULL handle");
  if (!B->have_solution) return fail(HOBI_ERR_STATE, "no solution: call hobi_solve_batch first");
  int64_t total = 0;
  for (hobi_t h : B->subs) total += h->nc;
  if (total == 0) return HOBI_OK;
  if (!forces) return fail(HOBI_ERR_ARG, "forces is NULL");
  DeviceGuard guard(B->device);
  for (int i = 0; i < B->nmol; ++i) {
    hobi_t h = B->subs[i];
    h->precision = B->precision;
    HOBI_CK(cudaMemcpyAsync(h->x, B->x + B->mols_h[i].u_off, sizeof(double) * 2 * h->nv, cudaMemcpyDeviceToDevice,
                            B->stream));
  }
  HOBI_CK(cudaStreamSynchronize(B->stream));
  // every member's field and forces on its own stream, then the copies in molecule order
  for (hobi_t h : B->subs) {
    h->have_solution = true;
    if (h->nc == 0) continue;
    HOBI_TRY(h->enter());
    HOBI_TRY(h->ensure_point_buffers(h->nc));
    HOBI_TRY(h->field_dev(h->nc, h->ctgt32, h->ctgt64, h->fld_pts));
    HOBI_CK(launch_charge_forces((int)h->nc, h->Q, h->fld_pts, h->fld_pts, h->stream));
    h->launches += 1;
    HOBI_TRY(h->leave());
  }
  int64_t off = 0;
  for (hobi_t h : B->subs) {
    if (h->nc == 0) continue;
    HOBI_CK(cudaStreamSynchronize(h->stream));
    HOBI_TRY(h->check_farfield());
    HOBI_CK(cudaMemcpy(forces + 3 * off, h->fld_pts, sizeof(double) * 3 * h->nc, cudaMemcpyDeviceToHost));
    off += h->nc;
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
