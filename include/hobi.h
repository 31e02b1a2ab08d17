/*
 * hobi.h -- C ABI of the GB300 (sm_103a) HOBI-PB solver library (libhobi.so).
 *
 * The library solves the well-posed boundary integral form of the linear
 * Poisson-Boltzmann equation (W. Geng, "Parallel Higher-order Boundary
 * Integral Electrostatics Computation on Molecular Surfaces with Curved
 * Triangulation", Sec. 2.1, Eqs. (8)/(9)) on a closed triangulated
 * molecular surface, with curved elements built from vertex normals
 * (Sec. 2.2), 4-point quadrature on regular triangles, 16-point regularised
 * Gauss-Legendre quadrature on singular triangles (Sec. 2.3), GMRES, the
 * electrostatic solvation energy (Sec. 2.5, Eq. (23)), and the reaction
 * potential, reaction field and reaction-field forces it implies.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an int status (hobi_status); nothing throws across the
 *    ABI. On failure, hobi_last_error() returns a message (thread-local).
 *  - Units: lengths in Angstrom, charges in e, kappa in 1/Angstrom. The
 *    unknowns u = [phi; dphi/dnu] (2 N_v doubles: the N_v vertex potentials,
 *    then the N_v normal derivatives on the inside of the surface; with the LOBI-PB
 *    scheme the collocation points are the N_f face centroids instead, and every "n_v"
 *    below reads n_f) are in the
 *    units of the formulation (G = 1/(4 pi r)); multiply by HOBI_KCAL_PER_MOL_E
 *    for kcal/(mol e). Energies are kcal/mol.
 *  - Dielectric ratio: eps = eps2/eps1 (the paper prints eps1/eps2 after
 *    Eq. (10); only eps2/eps1 makes Eqs. (8)/(9) consistent with the jump
 *    condition). Source terms carry 1/eps1.
 *  - Array arguments (vertices, faces, normals, charges, u, Au, phi, dphi,
 *    points, potentials, fields, forces) are HOST pointers when opt.mem_device == 0 and
 *    DEVICE pointers (on the handle's device) when opt.mem_device == 1.
 *    Scalar outputs (energy, info, counts) are always host pointers.
 *  - Work is ordered on opt.stream (a cudaStream_t; NULL = the legacy default
 *    stream). Calls return after their results are complete on that stream
 *    as far as host pointers are concerned; device-pointer outputs are
 *    complete in stream order.
 *  - A handle is not thread-safe: one thread at a time per handle. Different
 *    handles may be set up, used and destroyed from different threads at the
 *    same time (the library's shared state -- memory pool, pinned slots,
 *    autotuner cache -- is locked; a batch builds its molecules that way).
 */
#ifndef HOBI_H_
#define HOBI_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* 4 pi x 332.0716 kcal A/(mol e^2): formulation units -> kcal/(mol e). */
#define HOBI_KCAL_PER_MOL_E (4.0 * 3.14159265358979323846 * 332.0716)

typedef struct hobi_ctx* hobi_t;

typedef enum {
  HOBI_OK = 0,
  HOBI_ERR_ARG = -1,           /* bad argument (NULL, size, eps <= 0, kappa < 0, NaN) */
  HOBI_ERR_MESH = -2,          /* mesh not closed, not consistently oriented, bad index, degenerate */
  HOBI_ERR_CUDA = -3,          /* CUDA runtime error (message names the call) */
  HOBI_ERR_NOMEM = -4,         /* device allocation failed */
  HOBI_ERR_NOT_CONVERGED = -5, /* GMRES hit max_it; best iterate written, info filled */
  HOBI_ERR_BREAKDOWN = -6,     /* GMRES breakdown without convergence */
  HOBI_ERR_STATE = -7          /* call out of order (e.g. energy before a solve) */
} hobi_status;

typedef enum {
  HOBI_FP64 = 0,      /* every pair evaluation in IEEE double */
  HOBI_FP32_BULK = 1  /* far-field pair sums in FP32 with FP64 tile accumulation; FP64 for
                         setup, the singular-triangle correction, GMRES and the energy sum */
} hobi_precision;

typedef enum {
  HOBI_SCHEME_HOBI = 0, /* curved elements, 4-point regular + 16-point singular rules, unknowns at the
                           N_v vertices (Sec. 2.2-2.3) */
  HOBI_SCHEME_LOBI = 1  /* the paper's low-order comparison scheme LOBI-PB (Sec. 2.4, Eqs.
                           (21)/(22)): flat triangles, centroid collocation, the singular
                           (self) triangle dropped; unknowns at the N_f centroids, normals are the
                           flat face normals (vertex_normals are only validated) */
} hobi_scheme;

typedef struct {
  int32_t precision;  /* hobi_precision (default HOBI_FP32_BULK) */
  int32_t mem_device; /* 0: array arguments are host pointers; 1: device pointers */
  void* stream;       /* cudaStream_t the work is ordered on; NULL: legacy default stream */
  int32_t restart;    /* GMRES restart length m (default 50, max 200) */
  int32_t use_graph;  /* 1 (default): replay each GMRES iteration as a captured CUDA graph */
  int32_t device;     /* CUDA device ordinal; -1 (default): the current device */
  int32_t scheme;     /* hobi_scheme (default HOBI_SCHEME_HOBI); the batch API accepts HOBI only */
  int32_t autotune;   /* 1 (default): hobi_setup times the candidate FP32 far-field block shapes
                         (threads x targets per thread x source-tile size) on the problem and keeps
                         the fastest; decisions are cached per process by problem size, and in the
                         file named by the environment variable HOBI_AUTOTUNE_CACHE if set.
                         0: the analytic planner's choice. */
  int32_t ff_shape;   /* -1 (default): chosen as above; 0..3: use that FP32 block shape (see
                         hobi_plan_info) */
  int32_t fast_degree; /* 0 (default): the FP32 far field is summed directly over every node, as in
                          the paper. 2..10: fast summation by a barycentric Lagrange treecode of
                          this interpolation degree (beyond the paper, which names fast summation
                          as future work; see hobi_fast_info). FP32_BULK precision, HOBI scheme;
                          the FP64 path stays direct. In a batch, a molecule uses it when it has
                          at least 4096 collocation points and its plan needs at most 0.6 of the
                          direct pair evaluations; the others stay direct. */
  double fast_theta;   /* treecode admissibility parameter in (0, 1] (default 0.7): a source
                          cluster C of more than (n+1)^3 nodes acts on a target batch B through its
                          (n+1)^3 Chebyshev proxy points when r_B + r_C < theta |c_B - c_C| */
  int32_t gmres_scaling; /* 1 (default): GMRES works on the unknowns scaled by the inverse of the
                            diagonal coefficients (1/2)(1 + eps) and (1/2)(1 + 1/eps) of the two row
                            blocks of Eqs. (17)-(20) (right preconditioning by that constant diagonal;
                            the residual and the stopping test stay those of A u = b). The paper
                            states no scaling; its Table 3 reports 9-13 iterations for a protein,
                            which the scaled system reproduces on molecules and the unscaled one
                            (about three times as many) does not. 0: unscaled GMRES. */
} hobi_options;

typedef struct {
  int32_t iterations;    /* matvecs spent inside the Krylov iterations */
  int32_t converged;     /* 1 if ||b - A u|| / ||b|| <= tol (Givens estimate) */
  double rel_residual;   /* final relative residual estimate */
  double solve_ms;       /* wall time of hobi_solve on the handle's stream (CUDA events) */
  double farfield_pairs; /* target-source pair evaluations of the far field in the Krylov
                            iterations (iterations x pairs per matvec; the residual matvecs
                            of a warm start or restart are not counted) */
  double* resid_history; /* optional host buffer (caller-owned) for the residual after each it. */
  int32_t resid_capacity;/* length of resid_history (entries written: min(capacity, iterations+1)) */
} hobi_solve_info;

/* Fill *opt with the defaults listed in hobi_options. */
void hobi_default_options(hobi_options* opt);

/* Build a solver for one molecule (Sec. 2.6 routines (1)-(4)).
 *   vertices       [n_v][3] double, Angstrom.
 *   faces          [n_f][3] int32, 0-based vertex indices, counter-clockwise seen from outside
 *                  (the right-hand normal points out of the molecule).
 *   vertex_normals [n_v][3] double, outward; normalised by the callee.
 *   charges        [n_c][4] double: x, y, z (Angstrom), q (e). n_c may be 0 (charges NULL).
 *   eps1, eps2     interior / exterior dielectric constants (> 0); kappa >= 0 (1/A).
 *   opt            NULL for defaults.
 * Validates the mesh on the device (indices in range, distinct corners, every directed edge
 * matched by exactly one opposite edge, no unreferenced vertex, positive enclosed volume,
 * finite non-zero normals) and returns HOBI_ERR_MESH with a message otherwise.
 * Copies every input into library-owned device memory; the caller may free its arrays on
 * return. Then builds the curved elements and quadrature nodes, the vertex-to-face adjacency,
 * the singular-triangle correction table and the right-hand side [S1; S2] (Eq. (11)).
 * On success *out owns all device memory until hobi_destroy. */
int hobi_setup(const double* vertices, int64_t n_v, const int32_t* faces, int64_t n_f,
               const double* vertex_normals, const double* charges, int64_t n_c, double eps1,
               double eps2, double kappa, const hobi_options* opt, hobi_t* out);

/* Switch the far-field precision of later matvec/solve/energy calls (hobi_precision). */
int hobi_set_precision(hobi_t h, int32_t precision);

/* Sizes of the problem (any output pointer may be NULL). n_points: collocation points, i.e.
 * the length of phi / dphi and half the length of u (N_v for HOBI, N_f for LOBI); n_nodes:
 * source quadrature nodes (4 N_f for HOBI, N_f for LOBI). */
int hobi_sizes(hobi_t h, int64_t* n_v, int64_t* n_f, int64_t* n_c, int64_t* n_nodes, int64_t* n_points);

/* One discrete operator application Au = A u (Eqs. (17)-(20)): u and Au are 2 n_v
 * doubles (layout above). Au must not alias u. */
int hobi_matvec(hobi_t h, const double* u, double* Au);

/* Right-hand side b = [S1; S2] at the vertices (Eq. (11)), 2 n_v doubles. */
int hobi_rhs(hobi_t h, double* b);

/* Solve A u = b by GMRES from u = 0 (restart opt.restart) until ||b - A u||/||b|| <= tol or
 * max_it matvecs. Writes phi (n_v) and dphi (n_v) -- either may be NULL -- and keeps u in the
 * handle for hobi_energy. Returns HOBI_OK, HOBI_ERR_NOT_CONVERGED (best iterate written) or
 * HOBI_ERR_BREAKDOWN. info may be NULL. */
int hobi_solve(hobi_t h, double tol, int32_t max_it, double* phi, double* dphi,
               hobi_solve_info* info);

/* Mixed-precision solve (iterative refinement; the paper has no counterpart, it works in FP64):
 * starting from u = 0, each step forms the residual r = b - A u with the FP64 far field, stops when
 * ||r|| / ||b|| <= tol, and otherwise solves A d = r with FP32-bulk GMRES to 1e-6 (at most max_it
 * matvecs; fast summation when enabled) and sets u += d; at most max_refine corrections. The
 * result meets tol on the FP64 operator, which plain FP32-bulk GMRES cannot below ~1e-6, at
 * about one FP64 matvec per correction instead of one per Krylov iteration. The handle's
 * precision is unchanged on return. info: iterations = FP32 Krylov iterations in total,
 * rel_residual = the final FP64 residual, resid_history = the FP64 residual after each step
 * (first entry 1). Returns HOBI_OK or HOBI_ERR_NOT_CONVERGED (u written either way). */
int hobi_solve_refined(hobi_t h, double tol, int32_t max_refine, int32_t max_it, double* phi, double* dphi,
                       hobi_solve_info* info);

/* Warm start / resume: as hobi_solve, but GMRES starts from x0 = u0 (2 n_v doubles) or, when u0
 * is NULL, from the handle's current solution (a previous solve or hobi_set_solution; else
 * HOBI_ERR_STATE). The stopping test stays ||b - A u|| / ||b|| <= tol, so resuming a solve that
 * stopped at a loose tolerance continues it, and a converged u0 returns after 0 iterations. The
 * paper has no counterpart (its GMRES starts from an unstated guess). */
int hobi_solve_from(hobi_t h, const double* u0, double tol, int32_t max_it, double* phi, double* dphi,
                    hobi_solve_info* info);

/* Replace the handle's solution by u (2 n_v doubles), e.g. to evaluate the energy of a given
 * surface potential. */
int hobi_set_solution(hobi_t h, const double* u);

/* Copy the handle's solution u (2 n_v doubles) out. */
int hobi_get_solution(hobi_t h, double* u);

/* Reaction potential phi_reac at n_points points inside the molecule (the integral part of
 * Eq. (23), regular rule on every element), from the handle's solution.
 * points [n_points][3], phi [n_points] (formulation units). */
int hobi_reaction_potential(hobi_t h, const double* points, int64_t n_points, double* phi);

/* Reaction field -grad phi_reac at n_points points off the surface: the gradient, with respect to
 * the point, of the reaction potential above (the same regular-rule sum, differentiated term by
 * term), from the handle's solution. The paper motivates accurate potentials and fields near the
 * interface (Sec. 1) but prints no field formula; with d = x - y, E = exp(-kappa r) and
 * P = E (1 + kappa r) each node contributes -[(P - 1) sigma d + (eps P - 1) m
 * - (kappa^2 eps E + 3 (eps P - 1)/r^2)(d . m) d]/r^3, the gradient of its (1 - E)/r sigma
 * + (eps P - 1)(d . m)/r^3 term.
 * points [n_points][3] (A), field [n_points][3] (formulation units per A), both in the memory
 * space of the handle's mem_device option. A point must not coincide with a quadrature node.
 * HOBI scheme only (HOBI_ERR_ARG for LOBI-PB); HOBI_ERR_STATE without a solution;
 * n_points == 0 returns HOBI_OK. */
int hobi_reaction_field(hobi_t h, const double* points, int64_t n_points, double* field);

/* Reaction-field force on every charge, 4 pi C q_k (-grad phi_reac)(x_k) with C = 332.0716: the
 * force of the polarised solvent on charge k with the dielectric surface held fixed, in
 * kcal/(mol A) (the units of E_sol of Eq. (23) per A). The paper computes energies only; for a
 * fixed surface this is minus the gradient of E_sol with respect to x_k.
 * forces [n_c][3], in the memory space of the handle's mem_device option. HOBI scheme only;
 * HOBI_ERR_STATE without a solution; a handle without charges returns HOBI_OK. */
int hobi_reaction_forces(hobi_t h, double* forces);

/* Same result as hobi_reaction_potential, but the call allocates no device memory. The paper
 * has no counterpart. It is meant for callers that must not allocate once they are running: a
 * host whose device memory is owned by another allocator (a framework's caching pool holding the
 * GPU's free memory, where a cudaMalloc from this library would fail or upset the pool's
 * accounting), a service whose device-memory footprint is fixed at start-up, or a latency-bound
 * loop that cannot pay cudaMalloc's cost and its synchronisation with the device's other streams.
 * Create the handle (hobi_setup) beforehand; this call then uses the handle's tables plus one
 * file-scope device array of 2.5 MiB that every GPU loading the library keeps until process exit.
 *   n_points <= 4096 per call; larger requests return HOBI_ERR_ARG (split them, or use
 *   hobi_reaction_potential). n_points == 0 returns HOBI_OK and touches nothing.
 *   points/phi follow opt.mem_device like every array argument.
 *   The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 *   and keeps it for the later calls.
 *   The array is shared by every call on a device and keeps the last call's contents (each call
 *   overwrites every entry it reads, so nothing needs clearing): calls that overlap on the GPU
 *   (different streams or handles on one device) race on it.
 *   With hobi_profile_enable on, its far-field launch is timed like the others.
 * Results equal hobi_reaction_potential's up to summation order (at most 64 source chunks). */
int hobi_reaction_potential_noalloc(hobi_t h, const double* points, int64_t n_points, double* phi);

/* Electrostatic solvation energy E_sol = (1/2) sum_k q_k phi_reac(x_k) in kcal/mol
 * (Eq. (23)) from the handle's solution; requires hobi_solve or
 * hobi_set_solution first (else HOBI_ERR_STATE). e_sol is a host pointer. */
int hobi_energy(hobi_t h, double* e_sol);

/* Debug/parity accessors (host or device pointers per mem_device, FP64):
 * quadrature nodes of the regular rule, [n_f][4][3] each: position y_{j,m}, unit normal
 * nu_{j,m}, and W_{j,m,n} = w_m J_{j,m} L_n(r_m, s_m) (Sec. 2.2, Eq. (17)). */
int hobi_get_nodes(hobi_t h, double* y, double* nu, double* W);

/* Singular-triangle correction table: one entry per (vertex i, face j incident to i), in
 * vertex order then ascending face index. For entry e: vertex[e] = i, face[e] = j, and
 * coeff[e][n][k] (k = K1..K4) = (16-point singular rule) - (4-point regular rule) of
 * sum_m W_{j,m,n} K_k(x_i, y_{j,m}) (Sec. 2.3, Eqs. (19)/(20) minus Eqs. (17)/(18)).
 * Call with all three arrays NULL to get *n_entries first. Arrays are HOST pointers. */
int hobi_get_correction(hobi_t h, int64_t* n_entries, int32_t* vertex, int32_t* face,
                        double* coeff);

/* Far-field kernel timing for roofline measurement: when enabled, CUDA events are recorded
 * on the launching stream around every far-field launch (inside the captured GMRES graph as
 * event-record nodes when graphs are in use); hobi_profile_read returns the summed kernel
 * milliseconds, the number of launches and the pair evaluations they did, and resets the
 * counters. */
int hobi_profile_enable(hobi_t h, int32_t on);
int hobi_profile_read(hobi_t h, double* farfield_ms, int64_t* launches, double* pairs);

/* Number of CUDA kernels this handle has launched since hobi_setup began (setup included;
 * a replayed GMRES graph counts each of its kernels). */
int hobi_kernel_launches(hobi_t h, int64_t* n);

/* The FP32 far-field launch plan of the matvec: block shape index (0: 32 threads x 8 targets,
 * 128-node tiles; 1: 64 x 8, 128; 2: 32 x 8, 64; 3: 32 x 4, 64), source chunks, and whether
 * the shape was measured by the autotuner (1) or chosen analytically (0). */
int hobi_plan_info(hobi_t h, int32_t* shape, int32_t* chunks, int32_t* tuned);

/* Fast summation (options.fast_degree > 0; no counterpart in the paper, which sums the far field
 * directly and names fast summation as future work). The treecode is planned once in hobi_setup:
 * an octree over the regular-rule nodes (leaves of at most 256 nodes), target batches of 256
 * vertices (recursive splits along the longest box axis) and, per batch, the source clusters
 * summed directly and those replaced by their (n+1)^3 Chebyshev proxy points. Reports, per
 * matvec, the pair evaluations with nodes (direct_pairs) and with proxy points (approx_pairs),
 * and the numbers of batches, proxy clusters and evaluation tasks. All zero when fast summation
 * is off. Any pointer may be NULL. */
int hobi_fast_info(hobi_t h, int64_t* direct_pairs, int64_t* approx_pairs, int32_t* batches,
                   int32_t* proxy_clusters, int32_t* tasks);

/* The same statistics for a treecode plan built on the host from given FP64 points, without a
 * handle or a GPU: nodes [n_nodes][3] (sources), targets [n_targets][3], both host arrays. Plan
 * inspection for callers choosing degree and theta before a setup. */
int hobi_fast_plan_stats(const double* nodes, int64_t n_nodes, const double* targets, int64_t n_targets,
                         int32_t degree, double theta, int64_t* direct_pairs, int64_t* approx_pairs,
                         int32_t* batches, int32_t* proxy_clusters);

/* Accuracy accessor of the FP64 far field's own pair functions, evaluated on the current CUDA
 * device: rsqrt_x[k] = 1/sqrt(x[k]) (MUFU seed + one Newton step) and exp_neg_x[k] = exp(-x[k])
 * (256-entry table of 2^(j/256) + degree-4 polynomial), exactly as the FP64 kernels compute
 * 1/r and e^{-kappa r} (kernels of Eq. (10) in the paper). x: n host doubles in [0, 1e12]
 * (x = 0 gives rsqrt inf; far-field arguments stay below 1e7); n <= 2^24. All three arrays
 * are HOST arrays. Allocates and frees temporary device memory. */
int hobi_fp64_pair_functions(const double* x, int64_t n, double* rsqrt_x, double* exp_neg_x);

/* Failure-path check of the far-field source-tile pipeline (no counterpart in the paper). The
 * far-field kernels wait for each bulk-copied source tile on a shared-memory barrier, and every
 * wait is bounded: after about a second without the copy's arrival the kernel sets the handle's
 * error flag, drains its own copies and returns, and the call that launched it returns
 * HOBI_ERR_CUDA ("far-field source-tile pipeline timed out"). This call exercises that path
 * without faulting anything: one warp, on the handle's stream, initialises the tile barriers as
 * the kernels do and waits on a phase that no copy will complete. Expected result: HOBI_ERR_CUDA
 * with that message after about one second (*elapsed_ms, nullable host pointer, receives the
 * kernel's duration); the flag is then cleared and the handle stays usable. */
int hobi_check_tile_wait_timeout(hobi_t h, double* elapsed_ms);

/* Free every resource of the handle (NULL is a no-op). Its device memory goes back to the
 * library's stream-ordered memory pool for that device, which keeps it for the next handle
 * (setting up a handle then costs no cudaMalloc, destroying one no device-wide cudaFree) and
 * holds it until the process exits. */
void hobi_destroy(hobi_t h);

/* ---------------------------------------------------------------------------------------
 * Batched solve: many molecules (same eps1, eps2, kappa) solved together. Every GMRES step
 * runs one far-field launch over a task list covering every unconverged molecule,
 * and the Arnoldi/Givens work of all molecules in one set of launches (replayed as a CUDA
 * graph); converged molecules drop out. Each molecule follows exactly the single-molecule
 * method above (Sec. 2.2-2.3, Eqs. (17)-(20)), with its own Krylov space, residual
 * test and restart.
 * ------------------------------------------------------------------------------------- */
typedef struct hobi_batch_ctx* hobi_batch_t;

/* Molecule m owns rows [vertex_offsets[m], vertex_offsets[m+1]) of vertices/vertex_normals,
 * [face_offsets[m], face_offsets[m+1]) of faces (0-based indices LOCAL to molecule m's
 * vertices) and [charge_offsets[m], charge_offsets[m+1]) of charges. The three offset arrays
 * (n_mol + 1 int64 each, starting at 0) are HOST arrays; the data arrays follow opt.mem_device.
 * Per-molecule errors are reported as for hobi_setup, prefixed with the molecule index. */
int hobi_setup_batch(int32_t n_mol, const double* vertices, const int64_t* vertex_offsets,
                     const int32_t* faces, const int64_t* face_offsets, const double* vertex_normals,
                     const double* charges, const int64_t* charge_offsets, double eps1, double eps2,
                     double kappa, const hobi_options* opt, hobi_batch_t* out);

/* n_mol, total vertices (sum of n_v) and total quadrature nodes (any pointer may be NULL). */
int hobi_batch_sizes(hobi_batch_t b, int32_t* n_mol, int64_t* total_vertices, int64_t* total_nodes);

int hobi_batch_set_precision(hobi_batch_t b, int32_t precision);

/* Au = A u for every molecule; u and Au are the concatenation of the molecules' 2 n_v blocks
 * ([phi_m; dphi_m] in molecule order). */
int hobi_matvec_batch(hobi_batch_t b, const double* u, double* Au);

/* GMRES for every molecule (tol, max_it and the restart length apply per molecule).
 * phi, dphi: sum n_v doubles each, molecule blocks at vertex_offsets (either may be NULL).
 * iterations, status: n_mol entries each (HOST, may be NULL): Krylov iterations and
 * HOBI_OK / HOBI_ERR_NOT_CONVERGED / HOBI_ERR_BREAKDOWN per molecule. info (nullable)
 * aggregates: batched steps, all converged, worst residual, solve time, pair evaluations.
 * Returns HOBI_OK when every molecule converged. */
int hobi_solve_batch(hobi_batch_t b, double tol, int32_t max_it, double* phi, double* dphi,
                     int32_t* iterations, int32_t* status, hobi_solve_info* info);

/* Solvation energy of every molecule (Eq. (23)), e_sol[n_mol] HOST, kcal/mol. */
int hobi_energy_batch(hobi_batch_t b, double* e_sol);

/* Reaction-field force on every charge of every molecule, as hobi_reaction_forces:
 * forces [sum n_c][3] HOST, kcal/(mol A), molecule blocks at charge_offsets. */
int hobi_reaction_forces_batch(hobi_batch_t b, double* forces);

/* Timing of the batched far-field launches, as hobi_profile_enable / hobi_profile_read
 * (pairs counts only the molecules still iterating at each launch; for a molecule on fast
 * summation, its node and proxy pair evaluations; the timed span includes the treecode's
 * upward pass). */
int hobi_batch_profile_enable(hobi_batch_t b, int32_t on);
int hobi_batch_profile_read(hobi_batch_t b, double* farfield_ms, int64_t* launches, double* pairs);

/* CUDA kernels launched by the batch handle and its per-molecule tables since setup. */
int hobi_batch_kernel_launches(hobi_batch_t b, int64_t* n);

void hobi_destroy_batch(hobi_batch_t b);

/* Message of the last failing call on this thread ("" if none). */
const char* hobi_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HOBI_H_ */
