// hobi_capi.cu -- the C ABI declared in include/hobi.h for one molecule: handle lifetime, device
// memory, stream ordering, the setup pipeline, the matvec pipeline, the GMRES driver (optionally
// replayed from a captured CUDA graph), the energy and the off-surface potential. The batched
// handle is in hobi_batch.cu; the pieces both share are in hobi_host.cuh.
#include "hobi_host.cuh"

namespace hobi {
namespace host {
thread_local std::string g_err;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};
std::mutex g_pinned_mu;
std::vector<void*> g_pinned_free;
}  // namespace

cudaError_t pool_alloc(void** p, size_t bytes, int device, cudaStream_t s) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[device]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = device;
      cudaMemPool_t created = nullptr;
      cudaError_t e = cudaMemPoolCreate(&created, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = UINT64_MAX;  // hold freed memory for the next handle
      e = cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) {
        cudaMemPoolDestroy(created);
        return e;
      }
      g_pool[device] = created;
    }
    pool = g_pool[device];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t pool_free(void* p, cudaStream_t s) { return cudaFreeAsync(p, s); }

cudaError_t DeviceArena::get(void** p, size_t bytes, cudaStream_t s) {
  constexpr size_t kAlign = 256;
  bytes = (bytes + kAlign - 1) / kAlign * kAlign;
  std::unique_lock<std::mutex> lock(mu, std::defer_lock);
  if (shared) lock.lock();
  const cudaStream_t as = shared ? home : s;
  auto new_block = [&](void** q, size_t n) {
    cudaError_t e = pool_alloc(q, n, device, as);
    if (e == cudaSuccess && shared) e = cudaStreamSynchronize(home);
    return e;
  };
  if (bytes >= direct) {
    cudaError_t e = new_block(p, bytes);
    if (e == cudaSuccess) own.push_back(*p);
    return e;
  }
  if (bytes > left) {
    void* c = nullptr;
    cudaError_t e = new_block(&c, chunk);
    if (e != cudaSuccess) return e;
    chunks.push_back(c);
    cur = static_cast<char*>(c);
    left = chunk;
  }
  *p = cur;
  cur += bytes;
  left -= bytes;
  return cudaSuccess;
}

void DeviceArena::put(void* p, cudaStream_t s) {
  std::unique_lock<std::mutex> lock(mu, std::defer_lock);
  if (shared) lock.lock();
  for (size_t i = 0; i < own.size(); ++i)
    if (own[i] == p) {
      pool_free(p, s);
      own.erase(own.begin() + i);
      return;
    }
}

void DeviceArena::release_all(cudaStream_t s) {
  std::unique_lock<std::mutex> lock(mu, std::defer_lock);
  if (shared) lock.lock();
  for (void* b : chunks) pool_free(b, s);
  for (void* b : own) pool_free(b, s);
  chunks.clear();
  own.clear();
  cur = nullptr;
  left = 0;
}

void* pinned_slot() {
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  if (g_pinned_free.empty()) {
    constexpr int kSlots = 64;
    void* slab = nullptr;
    if (cudaMallocHost(&slab, kSlots * kPinnedSlot) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int k = kSlots - 1; k >= 0; --k) g_pinned_free.push_back(static_cast<char*>(slab) + k * kPinnedSlot);
  }
  void* q = g_pinned_free.back();
  g_pinned_free.pop_back();
  return q;
}

void pinned_slot_free(void* p) {
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  g_pinned_free.push_back(p);
}

}  // namespace host
}  // namespace hobi

namespace hobi {
namespace host {

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

}  // namespace host
}  // namespace hobi

namespace {

constexpr int kTuneLaunches = 4;  // per candidate shape: one warm-up, then the fastest of three

// Autotuner decisions, per process (and optionally in a file): key -> shape
std::mutex g_tune_mu;
std::vector<std::pair<std::string, int>> g_tune;
bool g_tune_loaded = false;

// The device's name, read once per device (cudaGetDeviceProperties queries every attribute).
std::string device_name(int device) {
  static std::mutex mu;
  static std::vector<std::string> names;
  std::lock_guard<std::mutex> lock(mu);
  if (device < 0) return "gpu";
  if ((size_t)device >= names.size()) names.resize(device + 1);
  if (names[device].empty()) {
    cudaDeviceProp prop;
    std::string name = cudaGetDeviceProperties(&prop, device) == cudaSuccess ? prop.name : "gpu";
    for (char& c : name)
      if (c == ' ') c = '_';
    names[device] = name;
  }
  return names[device];
}

std::string tune_key(int device, int scheme, int64_t nv, int64_t n_pad) {
  return device_name(device) + " " + std::to_string(scheme) + " " + std::to_string(nv) + " " + std::to_string(n_pad);
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
  h->host_scalar = static_cast<double*>(pinned_slot());
  if (!h->host_scalar) return fail(HOBI_ERR_NOMEM, "pinned host slot allocation failed");
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
  if (h->gmres_scaling) {  // D^-1 per unknown (inverse diagonal coefficients) and the scaled Arnoldi vector
    HOBI_TRY(h->alloc(&h->dscale, n));
    HOBI_TRY(h->alloc(&h->zvec, n));
    HOBI_CK(launch_fill_scale(h->dscale, h->nv, 1.0 / (0.5 * (1.0 + h->eps)), 1.0 / (0.5 * (1.0 + 1.0 / h->eps)),
                              h->stream));
    h->launches += 1;
  }
  HOBI_TRY(h->alloc(&h->hcol, m + 1));
  HOBI_TRY(h->alloc(&h->cvec, m + 1));
  HOBI_TRY(h->alloc(&h->nrm, 1));
  HOBI_TRY(h->alloc(&h->dpart, (size_t)(m + 1) * kDotBlocks));
  HOBI_TRY(h->alloc(&h->st, 1));
  static_assert(sizeof(GmresState) <= kPinnedSlot, "GMRES state read-back must fit a pinned slot");
  h->st_host = static_cast<GmresState*>(pinned_slot());
  if (!h->st_host) return fail(HOBI_ERR_NOMEM, "pinned host slot allocation failed");
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
  opt->gmres_scaling = 1;
}

const char* hobi_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace hobi {
namespace host {
int create_handle(const double* vertices, int64_t n_v, const int32_t* faces, int64_t n_f, const double* vertex_normals,
                  const double* charges, int64_t n_c, double eps1, double eps2, double kappa, const hobi_options* opt,
                  bool light, hobi_t* out, DeviceArena* arena) {
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
  if (o.gmres_scaling != 0 && o.gmres_scaling != 1) return fail(HOBI_ERR_ARG, "gmres_scaling must be 0 or 1");

  int dev = o.device;
  if (dev < 0) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HOBI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  DeviceGuard guard(dev);
  hobi_ctx* h = new hobi_ctx();
  h->device = dev;
  h->own_arena.device = dev;
  if (arena) h->arena = arena;
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
  h->gmres_scaling = o.gmres_scaling;
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
    r = host_guard([&] { return setup_impl(h, vertices, faces, vertex_normals, charges, light); });
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
// Eq. (23): the reaction potential at the charges and the weighted sum, queued on the handle's
// stream with the scalar's copy to pinned host memory; energy_finish waits and reads it. Split so
// that a batch can queue all its members before waiting for any.
int energy_enqueue(hobi_ctx* h) {
  if (h->nc == 0) return HOBI_OK;
  HOBI_TRY(h->enter());
  HOBI_TRY(h->ensure_point_buffers(h->nc));
  HOBI_TRY(h->reaction_dev(h->nc, h->ctgt32, h->ctgt64, h->phi_pts));
  HOBI_CK(launch_energy_sum((int)h->nc, h->Q, h->phi_pts, h->e_dev, h->stream));
  h->launches += 1;
  HOBI_CK(cudaMemcpyAsync(h->host_scalar, h->e_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return h->leave();
}

int energy_finish(hobi_ctx* h, double* e_sol) {
  if (h->nc == 0) {
    *e_sol = 0.0;
    return HOBI_OK;
  }
  HOBI_CK(cudaStreamSynchronize(h->stream));
  HOBI_TRY(h->collect_profile());
  HOBI_TRY(h->check_farfield());
  *e_sol = *h->host_scalar;
  return HOBI_OK;
}
}  // namespace host
}  // namespace hobi

extern "C" {

int hobi_setup(const double* vertices, int64_t n_v, const int32_t* faces, int64_t n_f, const double* vertex_normals,
               const double* charges, int64_t n_c, double eps1, double eps2, double kappa, const hobi_options* opt,
               hobi_t* out) {
  NvtxRange nvtx_range("hobi_setup");
  return host_guard([&] {
    return create_handle(vertices, n_v, faces, n_f, vertex_normals, charges, n_c, eps1, eps2, kappa, opt, false, out);
  });
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
    HOBI_CK(launch_finish_cycle(h->H, m, h->g, h->st, h->y, h->Vb, n, h->x, n, h->dscale, h->stream));
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
  return host_guard([&] { return solve_impl(h, nullptr, false, tol, max_it, phi, dphi, info); });
}

int hobi_solve_refined(hobi_t h, double tol, int32_t max_refine, int32_t max_it, double* phi, double* dphi,
                       hobi_solve_info* info) {
  NvtxRange nvtx_range("hobi_solve_refined");
  return host_guard([&] { return solve_refined_impl(h, tol, max_refine, max_it, phi, dphi, info); });
}

int hobi_solve_from(hobi_t h, const double* u0, double tol, int32_t max_it, double* phi, double* dphi,
                    hobi_solve_info* info) {
  NvtxRange nvtx_range("hobi_solve_from");
  return host_guard([&] { return solve_impl(h, u0, true, tol, max_it, phi, dphi, info); });
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

int hobi_reaction_field(hobi_t h, const double* points, int64_t n_points, double* field) {
  NvtxRange nvtx_range("hobi_reaction_field");
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (n_points < 0 || (n_points > 0 && (!points || !field))) return fail(HOBI_ERR_ARG, "bad points/field arguments");
  if (h->scheme != HOBI_SCHEME_HOBI) return fail(HOBI_ERR_ARG, "the reaction field supports the HOBI scheme only");
  if (!h->have_solution) return fail(HOBI_ERR_STATE, "no solution: call hobi_solve or hobi_set_solution first");
  if (n_points == 0) return HOBI_OK;
  if (n_points > (int64_t(1) << 28)) return fail(HOBI_ERR_ARG, "too many points");
  DeviceGuard guard(h->device);
  HOBI_TRY(h->enter());
  HOBI_TRY(h->ensure_point_buffers(n_points));
  HOBI_TRY(h->copy_in(h->pts_in, points, 3 * n_points));
  HOBI_CK(launch_points((int)n_points, h->pts_in, 3, h->center, h->xs, h->ptgt32, h->ptgt64, h->stream));
  h->launches += 1;
  HOBI_TRY(h->field_dev(n_points, h->ptgt32, h->ptgt64, h->fld_pts));
  HOBI_TRY(h->copy_out(field, h->fld_pts, 3 * n_points));
  HOBI_TRY(h->finish());
  return h->check_farfield();
}

int hobi_reaction_forces(hobi_t h, double* forces) {
  NvtxRange nvtx_range("hobi_reaction_forces");
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  if (h->scheme != HOBI_SCHEME_HOBI) return fail(HOBI_ERR_ARG, "the reaction forces support the HOBI scheme only");
  if (!h->have_solution) return fail(HOBI_ERR_STATE, "no solution: call hobi_solve or hobi_set_solution first");
  if (h->nc == 0) return HOBI_OK;
  if (!forces) return fail(HOBI_ERR_ARG, "forces is NULL");
  DeviceGuard guard(h->device);
  HOBI_TRY(h->enter());
  HOBI_TRY(h->ensure_point_buffers(h->nc));
  HOBI_TRY(h->field_dev(h->nc, h->ctgt32, h->ctgt64, h->fld_pts));
  HOBI_CK(launch_charge_forces((int)h->nc, h->Q, h->fld_pts, h->fld_pts, h->stream));
  h->launches += 1;
  HOBI_TRY(h->copy_out(forces, h->fld_pts, 3 * h->nc));
  HOBI_TRY(h->finish());
  return h->check_farfield();
}

int hobi_energy(hobi_t h, double* e_sol) {
  NvtxRange nvtx_range("hobi_energy");
  if (!h || !e_sol) return fail(HOBI_ERR_ARG, "NULL argument");
  if (!h->have_solution) return fail(HOBI_ERR_STATE, "no solution: call hobi_solve or hobi_set_solution first");
  DeviceGuard guard(h->device);
  HOBI_TRY(energy_enqueue(h));
  return energy_finish(h, e_sol);
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
  return host_guard([&] {
    FastPlanHost P;
    const double origin[3] = {0.0, 0.0, 0.0};
    build_fast_plan(nodes, (int)n_nodes, targets, (int)n_targets, origin, 1.0, degree, theta, 1, 0, &P);
    if (direct_pairs) *direct_pairs = P.direct_pairs;
    if (approx_pairs) *approx_pairs = P.approx_pairs;
    if (batches) *batches = (int32_t)P.batch.size();
    if (proxy_clusters) *proxy_clusters = (int32_t)P.pc_offset.size();
    return (int)HOBI_OK;
  });
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

int hobi_check_tile_wait_timeout(hobi_t h, double* elapsed_ms) {
  NvtxRange nvtx_range("hobi_check_tile_wait_timeout");
  if (!h) return fail(HOBI_ERR_ARG, "NULL handle");
  DeviceGuard guard(h->device);
  HOBI_TRY(h->enter());
  HOBI_CK(cudaEventRecord(h->ev_t0, h->stream));
  HOBI_CK(launch_tile_wait_check(h->ff_err, h->stream));
  HOBI_CK(cudaEventRecord(h->ev_t1, h->stream));
  h->launches += 1;
  HOBI_TRY(h->leave());
  HOBI_CK(cudaEventSynchronize(h->ev_t1));
  if (elapsed_ms) {
    float ms = 0.f;
    HOBI_CK(cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1));
    *elapsed_ms = ms;
  }
  return h->check_farfield();
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

