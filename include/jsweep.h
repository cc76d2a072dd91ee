/*
 * jsweep.h — C ABI of a GB300 (sm_103a) library for the data-driven S_n
 * transport sweep of JSweep (arXiv 1803.09876).
 *
 * The method (Sec. II-C, Sec. V-A, Listing 1, and the source-iteration
 * algorithm of the appendix): for every ordinate direction Omega_m the mesh
 * induces a dependency graph on its cells — a cell may be solved only after
 * all of its upwind neighbours — and a sweep is a topological traversal of
 * that graph with a per-cell upwind solve at each vertex; the scalar flux
 * phi = sum_m w_m psi_m feeds the scattering source of the next source
 * iteration.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: JSWEEP_OK (0) or a negative
 *     JSWEEP_ERR_* code.  jsweep_last_error() returns a message describing the
 *     last failure of the calling thread (thread-local; valid until the next
 *     call on that thread).
 *   - Handles (mesh, quadrature, dags, batch) are opaque, owned by the library,
 *     and released by their *_destroy function.  Destroying NULL is a no-op.
 *   - Host input arrays are copied during the call; the caller keeps them.
 *   - "device" arrays are CUDA device pointers on the current device (for
 *     example torch.Tensor.data_ptr()); the caller allocates and owns them.
 *     Their element type is double for JSWEEP_F64 and float for JSWEEP_F32.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *     work is queued on it; calls that return host-visible results (counts,
 *     iteration numbers) synchronise that stream before returning.
 *   - Sizes and indices are int64 at the ABI; internally cell and face ids are
 *     int32, so n_cells and n_faces must be below 2^31.
 *   - Device memory the library needs for itself comes from the allocator set
 *     with jsweep_set_allocator (cudaMalloc/cudaFree by default).
 */
#ifndef JSWEEP_H
#define JSWEEP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define JSWEEP_API __attribute__((visibility("default")))
#else
#define JSWEEP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define JSWEEP_OK 0
#define JSWEEP_ERR_INVALID_ARG (-1)    /* bad pointer, size or option */
#define JSWEEP_ERR_MESH_INVALID (-2)   /* mesh failed validation (message names the id) */
#define JSWEEP_ERR_OOM (-3)            /* a device or host allocation failed */
#define JSWEEP_ERR_NOT_CONVERGED (-4)  /* source iteration hit max_iters (outputs filled) */
#define JSWEEP_ERR_DEVICE_TIMEOUT (-5) /* a bounded device-side wait ran out */
#define JSWEEP_ERR_CUDA (-6)           /* a CUDA runtime call failed */
#define JSWEEP_ERR_UNIMPLEMENTED (-7)  /* input outside what this build supports */
#define JSWEEP_ERR_CYCLE (-8)          /* a dependency cycle could not be broken */

/* ---- precisions ------------------------------------------------------- */
#define JSWEEP_F64 0 /* psi, phi, sources in double */
#define JSWEEP_F32 1 /* psi in float, phi in float with compensated sums; FP64 residual */

/* ---- sweep schedules (jsweep_options.sweep_mode) ----------------------- */
#define JSWEEP_MODE_AUTO 0       /* library picks */
#define JSWEEP_MODE_LEVEL_SYNC 1 /* one launch per level index, replayed from a CUDA graph */
#define JSWEEP_MODE_PERSISTENT 2 /* one grid-resident launch driven by dependency counters */
/* Patch programs (Sec. V-A, V-B): the cells are grouped into compact patches
 * of about patch_cells cells; one block runs a (patch, octant) program: it
 * stages the patch's geometry and sources in shared memory once and sweeps
 * every direction of the octant across the patch, layer by layer, waiting for
 * the values that enter the patch from upwind patches.  Programs are taken
 * from a device-wide queue; a direction whose inflow is not ready yet keeps
 * its progress and the program is queued again (the data-driven execution of
 * Listing 1 at patch granularity), so the schedule cannot deadlock. */
#define JSWEEP_MODE_PATCH 3

/* ---- schedule layers (jsweep_options.layering) ------------------------------
 * Both sweep schedules process the cells of a direction layer by layer; any
 * layering that increases along every dependency is valid and gives the same
 * results.  LEVEL uses the longest-path levels.  OCTANT (default) uses
 * kappa_m(c) = max(floor(rho_o * lambda_o(c)), 1 + max over upwind u of kappa_m(u)),
 * where lambda_o is the level of c for the diagonal direction of m's octant and
 * rho_o the largest level count of the octant over the diagonal's: the
 * directions of an octant then reach a cell at nearly the same time, so its
 * geometry and sources are fetched once for most of them. */
#define JSWEEP_LAYERS_OCTANT 0
#define JSWEEP_LAYERS_LEVEL 1

/* ---- work-unit orderings for the persistent schedule (jsweep_options.priority) */
#define JSWEEP_PRIO_LEVEL 0     /* by level index, all directions together */
#define JSWEEP_PRIO_DEPTH 1     /* by remaining depth: long directions start first */
#define JSWEEP_PRIO_OCTANT 2    /* level index staggered by octant */
/* Patch tasks (Sec. V-B patch-angle programs): the cells are cut into
 * contiguous id ranges ("patches"; the generated meshes number cells so that
 * a range is a spatial slab), and each (direction, patch) pair becomes one
 * task that a single resident warp runs from its first layer to its last, so
 * upwind values it wrote a moment ago are still in cache.  There are as many
 * patches as resident warps allow (directions x patches <= resident warps), so
 * every task is running at once and the sweep cannot deadlock whatever the
 * patch graph looks like.  Persistent schedule only (others treat it as
 * LEVEL); JSWEEP_ERR_UNIMPLEMENTED if the directions outnumber the resident
 * warps. */
#define JSWEEP_PRIO_PATCH 3
/* Patch tasks with SLBD vertex priority (Sec. V-D, Shortest Local Boundary
 * Distance): within every (direction, patch) task's layer, the units whose
 * cells lie closest to the patch's boundary (breadth-first distance in faces
 * to the nearest cell of another patch) run first, so the warps of the
 * neighbouring patches that wait on them are released sooner.  Same results
 * as every other order; persistent schedule only (others treat it as LEVEL). */
#define JSWEEP_PRIO_PATCH_SLBD 4

typedef struct jsweep_mesh_s *jsweep_mesh_t;
typedef struct jsweep_quad_s *jsweep_quad_t;
typedef struct jsweep_dags_s *jsweep_dags_t;
typedef struct jsweep_batch_s *jsweep_batch_t;

/* Options of the dependency-graph build and of the sweeps.  Zero or negative
 * numeric fields mean "default".  struct_size must be sizeof(jsweep_options). */
typedef struct {
    int struct_size;
    int sweep_mode;        /* JSWEEP_MODE_* */
    int priority;          /* JSWEEP_PRIO_*, persistent schedule only */
    int cluster_cells;     /* cells per work unit (vertex clustering grain, Sec. V-C); 1..32, default 32 */
    int blocks_per_sm;     /* persistent schedule: resident blocks per SM (default: occupancy) */
    int octant_stagger;    /* JSWEEP_PRIO_OCTANT: levels between octant starts (default: auto) */
    double spin_timeout_s; /* bounded device waits give up after this long (default 2 s) */
    int cycle_search_max;  /* cells a local cycle search may visit (default 256, max 1024) */
    int debug_block_waits; /* test hook, 0 in normal use: when nonzero every dependency wait of the
                              persistent schedule needs one more finished unit than can exist, so
                              the waits run out and the call returns JSWEEP_ERR_DEVICE_TIMEOUT */
    int layering;          /* schedule layers (set at jsweep_build_dags): JSWEEP_LAYERS_OCTANT (default)
                              or JSWEEP_LAYERS_LEVEL; results do not depend on it */
    int angles_per_warp;   /* data-driven schedule: units one warp runs side by side (1, 2 or 4; 0 =
                              1); each holds up to 32 / angles_per_warp cells of one direction */
    int unit_order;        /* order of the work units inside a layer: 0 = direction by direction,
                              1 = interleaved across the directions of an octant (default), so that
                              units covering the same cells for different directions run side by side
                              and share the cells' geometry and sources in cache */
    int patch_cells;       /* JSWEEP_MODE_PATCH: target cells per patch (default 512, 32..4096) */
    int eager_search_max;  /* cells a cycle search may visit while its direction is still peeling (default
                              64, at most cycle_search_max); a stalled direction searches up to
                              cycle_search_max, and a build that cannot break a cycle this way is
                              repeated once with cycle_search_max everywhere.  Lags do not depend on it. */
    int no_face_stream;    /* level-synchronous sweeps: 0 (default) reads each direction's face coefficients
                              (Omega.A per face and the upwind neighbours, one record per cell-direction in
                              sweep order, built at the handle's first such sweep: N x M x 32..96 bytes) as
                              a sequential stream; nonzero computes them from the cell geometry in the
                              sweep.  Results are bit-identical either way.  Once built, the stream stays
                              with the handle until it is destroyed (batches on the handle may read it). */
    int tail_units;        /* level-synchronous sweeps with the face stream and JSWEEP_PRIO_LEVEL: > 0 runs
                              the last slots that each hold fewer than this many work units in one launch
                              of one block per direction (the tail), each block sweeping its direction's
                              remaining layers in order with a block barrier between layers, instead of
                              one launch per slot; 0 (default) = no tail.  Results are bit-identical. */
    int no_sweep_order_psi; /* level-synchronous sweeps with the face stream: 0 (default) keeps a second copy
                              of psi in each direction's sweep order ([M][N][R], N x M x R x element bytes;
                              built at the first such sweep, kept with the handle) beside the cell-major
                              psi.  A slot then writes its cell-directions as one contiguous run and reads
                              its upwind values from the runs of the layers just before it, which stay in
                              L2; the face stream holds upwind positions in that order instead of cell
                              ids.  Nonzero reads upwind values from the cell-major psi.  Results are
                              bit-identical either way. */
} jsweep_options;

/* Fill *opt with defaults. */
JSWEEP_API int jsweep_options_default(jsweep_options *opt);

/* Message of the calling thread's last failure ("" if none). */
JSWEEP_API const char *jsweep_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
JSWEEP_API int jsweep_version(void);

/* Route the library's own device allocations through the caller's allocator
 * (for example PyTorch's caching allocator).  alloc returns a device pointer
 * or NULL; free releases one.  Both are called on the host thread making the
 * library call; stream is the stream the memory will first be used on.
 * Passing NULL for both restores cudaMalloc/cudaFree.  Memory obtained before
 * the switch is released with the allocator that produced it, so a free
 * function (and its ctx) must stay callable until every buffer it may release
 * is gone: until the handles and batch problems created while it was
 * installed are destroyed. */
typedef void *(*jsweep_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*jsweep_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
JSWEEP_API int jsweep_set_allocator(jsweep_alloc_fn alloc, jsweep_free_fn free_fn, void *ctx);

/* ---- mesh ----------------------------------------------------------------
 * A mesh of n_cells polyhedral cells and n_faces faces (Sec. II-B: the patch
 * holds cells and their adjacency; here one patch holds the whole mesh).
 *   face_cells [n_faces][2] (host): cell0, cell1 of each face; cell1 = -1 marks
 *     a boundary face.  The face id is the row index; it is the tie-break key
 *     of the cycle rule and the summation order of a cell's faces.
 *   normals [n_faces][3] (host): unit normal pointing from cell0 into cell1
 *     (outward from cell0 on a boundary face).
 *   areas [n_faces], volumes [n_cells] (host): positive.
 * Validation (JSWEEP_ERR_MESH_INVALID, message names the first offending id):
 * ids in range, cell0 != cell1, positive areas and volumes, unit normals
 * (|1-|n|| <= 1e-6), at most 7 faces per cell, at least one face per cell,
 * and closed cells: |sum_f +-a_f n_f| <= 1e-8 * sum_f a_f.
 * Boundary faces are numbered 0..n_bfaces-1 in increasing face id; inflow
 * arrays use that numbering. */
JSWEEP_API int jsweep_mesh_create(int64_t n_cells, int64_t n_faces, const int64_t *face_cells,
                       const double *normals, const double *areas, const double *volumes,
                       jsweep_mesh_t *out);
JSWEEP_API int jsweep_mesh_destroy(jsweep_mesh_t mesh);
JSWEEP_API int jsweep_mesh_info(jsweep_mesh_t mesh, int64_t *n_cells, int64_t *n_faces, int64_t *n_bfaces,
                     int *max_faces_per_cell);

/* ---- quadrature ------------------------------------------------------------
 * jsweep_quadrature_product (host only) fills the product set "n_polar
 * Gauss-Legendre polar cosines x n_azim azimuths per octant" (M = 8 n_polar
 * n_azim directions; weights sum to 4 pi):
 *   mu_i = the positive nodes, ascending, of the 2 n_polar-point
 *   Gauss-Legendre rule, weight w_i; phi_j = (j + 1/2)(pi/2)/n_azim, weight
 *   pi/(2 n_azim); Omega = (s_x sqrt(1-mu^2) cos phi, s_y sqrt(1-mu^2) sin phi,
 *   s_z mu); index m = octant*n_polar*n_azim + i*n_azim + j with octant bits
 *   (1, 2, 4) set for negative (x, y, z).
 *   dirs [M][3], weights [M] (host, caller-allocated).  1 <= n_polar, n_azim <= 64.
 * jsweep_quadrature_create copies any direction set (host arrays): directions
 * must be finite and non-zero (they need not be unit vectors: a 1D slab test
 * uses (mu, 0, 0)); weights finite. */
JSWEEP_API int jsweep_quadrature_product(int n_polar, int n_azim, double *dirs, double *weights);
JSWEEP_API int jsweep_quadrature_create(int64_t n_dirs, const double *dirs, const double *weights,
                             jsweep_quad_t *out);
JSWEEP_API int jsweep_quadrature_destroy(jsweep_quad_t quad);

/* ---- dependency graphs (Sec. V-A, Listing 1 init; cycle rule) -------------
 * Builds, on the device, for every direction m:
 *   - the upwind classification of every cell face from the FP64 sign of
 *     ((n_x O_x) + (n_y O_y)) + (n_z O_z) (no fused multiply-add);
 *   - the longest-path level of every cell (0 = no upwind neighbour);
 *   - cycle breaking: in every strongly connected component of two or more
 *     cells the active interior face of smallest id inside the component is
 *     lagged (its upwind value comes from the previous sweep), repeated until
 *     the graph is acyclic;
 *   - the level-major order (cells sorted by (level, cell id)) and the
 *     work-unit schedules of the sweeps.
 * The result is resident on the device and stays valid while mesh and quad
 * live (the handle keeps its own references).  Errors: JSWEEP_ERR_CYCLE if a
 * strongly connected component exceeds opt->cycle_search_max cells. */
JSWEEP_API int jsweep_build_dags(jsweep_mesh_t mesh, jsweep_quad_t quad, const jsweep_options *opt,
                      void *stream, jsweep_dags_t *out);
/* Releases the caller's reference; batch problems that use the handle keep it
 * alive until they are removed. */
JSWEEP_API int jsweep_dags_destroy(jsweep_dags_t dags);
/* n_dirs, the largest level count over directions, total lagged (face, dir) pairs. */
JSWEEP_API int jsweep_dags_info(jsweep_dags_t dags, int64_t *n_dirs, int64_t *max_levels, int64_t *n_lag_total);
JSWEEP_API int jsweep_dags_nlevels(jsweep_dags_t dags, int64_t m, int64_t *nlevels);
/* level_of_cell [n_cells] (host). */
JSWEEP_API int jsweep_dags_levels(jsweep_dags_t dags, int64_t m, int32_t *level_of_cell);
/* order [n_cells], level_ptr [nlevels+1] (host). */
JSWEEP_API int jsweep_dags_order(jsweep_dags_t dags, int64_t m, int32_t *order, int32_t *level_ptr);
/* The schedule the sweeps of direction m run: its layers (the octant-aligned
 * layers by default, the levels with JSWEEP_LAYERS_LEVEL; every active upwind
 * cell of a cell is in an earlier layer), as the number of layers in
 * *n_layers, the cells in layer-major order in order [n_cells] (host) and the
 * layer pointers in layer_ptr [n_layers+1] (host).  order and layer_ptr may be
 * NULL (then only the count is returned). */
JSWEEP_API int jsweep_dags_schedule(jsweep_dags_t dags, int64_t m, int64_t *n_layers, int32_t *order,
                                    int32_t *layer_ptr);
/* Lagged faces of direction m sorted by face id, rows (face, upwind cell,
 * downwind cell) into rows [*n][3] (host; may be NULL to query *n only). */
JSWEEP_API int jsweep_dags_lagged(jsweep_dags_t dags, int64_t m, int64_t *rows, int64_t *n);
/* Zero the lagged upwind values (the state a source iteration starts from). */
JSWEEP_API int jsweep_dags_reset_lag(jsweep_dags_t dags);
/* Replace the sweep options (mode, priority, grain, ...) of a built handle. */
JSWEEP_API int jsweep_dags_set_options(jsweep_dags_t dags, const jsweep_options *opt);

/* ---- one transport sweep (Listing 1 compute/solve; Sec. V-B) -------------
 * Sweeps all directions for nrhs right-hand sides with the step (upwind
 * finite-volume) scheme: for cell c and direction m, with mu_f a_f =
 * (Omega_m . n_f) a_f taken outward from c,
 *    psi = (S V + sum_{incoming f} |mu_f| a_f psi_up(f)) /
 *          (sigma_t V + sum_{outgoing f} mu_f a_f),
 * psi_up being the upwind cell's psi, the lagged value on a lagged face, or
 * the boundary inflow.  Then phi = sum_m w_m psi_m (FP32: compensated sum in
 * a fixed order, so results do not depend on the schedule).
 *   sigma_t [n_cells] (device), ang_source [nrhs][n_cells] (device, angular
 *   source per steradian), inflow [nrhs][n_bfaces] (device, isotropic boundary
 *   angular flux) or NULL for vacuum, phi_out [nrhs][n_cells] (device),
 *   psi_out [nrhs][n_dirs][n_cells] (device) or NULL.
 * Uses the handle's lagged values and then replaces them by this sweep's.
 * 1 <= nrhs <= 8.  Device-side waits are bounded (JSWEEP_ERR_DEVICE_TIMEOUT). */
JSWEEP_API int jsweep_sweep(jsweep_dags_t dags, int nrhs, int precision, const void *sigma_t,
                 const void *ang_source, const void *inflow, void *phi_out, void *psi_out,
                 void *stream);

/* ---- source iteration (appendix algorithm "Source iterative Sn solver") ---
 * phi^0 = 0, lagged values 0; repeat { S = (c sigma_t phi + q) / (4 pi);
 * sweep; residual r = max_c |phi_new - phi| / max_c |phi_new| per right-hand
 * side, in FP64 on the device } until r < tol for all right-hand sides.
 *   sigma_t, c_ratio [n_cells] (device; sigma_s = c_ratio * sigma_t),
 *   q [nrhs][n_cells] (device, total isotropic source), inflow as in
 *   jsweep_sweep, phi_out [nrhs][n_cells] (device).
 *   iters_out, resid_out (host, may be NULL): sweeps done, final residual.
 * Returns JSWEEP_ERR_NOT_CONVERGED (phi_out filled) after max_iters sweeps. */
JSWEEP_API int jsweep_source_iterate(jsweep_dags_t dags, int nrhs, int precision, const void *sigma_t,
                          const void *c_ratio, const void *q, const void *inflow, double tol,
                          int max_iters, void *phi_out, int *iters_out, double *resid_out,
                          void *stream);

/* ---- bounds-checked builds ----------------------------------------------------
 * A build with the flag JSWEEP_BOUNDS_CHECK (libjsweep_bounds.so, see the
 * package's build script) checks every gather index of the sweep kernels: cell
 * ids read from the orders, upwind cells, boundary faces, order positions and
 * directions.  The first index out of range on a device is recorded and its
 * access skipped (no trap).  Patch programs are not covered.
 *   jsweep_bounds_checked: 1 in such a build, 0 otherwise (no device work).
 *   jsweep_bounds_error: waits for the current device, then returns the
 *   recorded word in *word and clears it: 0 = none, else (code << 56) | index
 *   with code 1 cell id, 2 upwind cell, 3 boundary face, 4 order position,
 *   5 direction.  Always 0 in other builds. */
JSWEEP_API int jsweep_bounds_checked(void);
JSWEEP_API int jsweep_bounds_error(uint64_t *word);

/* ---- multigroup source iteration (the appendix's transport equation over
 * energy groups g and its source-iteration algorithm) -------------------------
 * phi^0 = 0, lagged values 0; repeat { S_g = (sum_h sigma_s[h][g] phi_h + q_g)
 * / (4 pi) for every group from the previous iterate of all groups; one sweep
 * per group with sigma_t[g] and the group's own lagged values; residual as in
 * jsweep_source_iterate, per group } until every group's residual < tol.
 *   n_groups G in 1..8; sigma_t [G][n_cells]; sigma_s [G][G][n_cells] with
 *   entry [h][g][c] the isotropic scattering rate from group h into group g in
 *   cell c (up- and downscatter allowed); q [G][n_cells] (total isotropic
 *   source); inflow [G][n_bfaces] or NULL for vacuum; phi_out [G][n_cells].
 *   All arrays are device arrays of the given precision.
 *   iters_out, resid_out (host, may be NULL): iterations, final residual.
 * Leaves the handle's lagged values at 0 (see jsweep_sweep).
 * Returns JSWEEP_ERR_NOT_CONVERGED (phi_out filled) after max_iters
 * iterations, JSWEEP_ERR_INVALID_ARG for a NULL array or G outside 1..8. */
JSWEEP_API int jsweep_source_iterate_mg(jsweep_dags_t dags, int n_groups, int precision, const void *sigma_t,
                             const void *sigma_s, const void *q, const void *inflow, double tol,
                             int max_iters, void *phi_out, int *iters_out, double *resid_out, void *stream);

/* ---- batches: many independent problems in one persistent launch ----------
 * Sec. V-B runs the (patch, angle) programs of all angles at once; a batch
 * extends that to many independent problems (meshes, direction sets,
 * right-hand sides, of uneven size): every source iteration sweeps all of the
 * batch's active problems in one data-driven launch.  Its work units (up to
 * 32 cells of one schedule layer of one direction of one problem) are merged
 * by schedule slot, so each problem's units stay in a topological order of
 * its graphs and the launch cannot deadlock.  The other steps of an iteration
 * (emission source, lagged-value copy, phi with the FP64 residual, the
 * convergence test) are batched kernels too, and the iteration is replayed
 * from a CUDA graph.  Every problem keeps its own state and stops on its own
 * test (residual below its tol, defined as for jsweep_source_iterate, or
 * max_iters); its phi is bit-identical to what jsweep_source_iterate returns
 * for it alone with the same precision and nrhs.
 *
 * Problems are identified by the id jsweep_batch_add returns (stable until
 * the problem is removed).  Problems may be added and removed between calls,
 * so a server can admit new requests while others are still iterating
 * (continuous batching).  A handle used by a batch problem stays alive until
 * the problem is removed, even if jsweep_dags_destroy is called meanwhile.
 * Calls on one batch must not overlap in time.
 *
 *   jsweep_batch_create: precision and nrhs shared by the batch's problems;
 *     opt (may be NULL) sets cluster_cells, angles_per_warp, unit_order,
 *     priority, spin_timeout_s, debug_block_waits, no_face_stream and
 *     no_sweep_order_psi of the batched launch.  A level-synchronous batch
 *     whose problems all have one face-slot count reads each handle's
 *     face-coefficient stream (built at the first step that needs it, kept with
 *     the handle and shared by every problem and sweep on it: N x M x 32..96
 *     bytes); with no_sweep_order_psi = 0 every problem also keeps a copy of its
 *     psi in sweep order (allocated by jsweep_batch_add) and the stream holds
 *     upwind positions, as in a single-problem sweep.  Otherwise it reads the
 *     cell geometry.  Results are bit-identical either way.
 *   jsweep_batch_problem_bytes: device bytes that jsweep_batch_add will
 *     allocate for a problem on this handle (its workspaces: psi, epoch flags,
 *     source records, lagged values, two phi buffers, inflow copy; not the
 *     handle's face-coefficient stream).
 *   jsweep_batch_add: a built handle and the problem's device arrays, laid out
 *     as for jsweep_source_iterate (sigma_t, c_ratio [N], q [nrhs][N], inflow
 *     [nrhs][n_bfaces] or NULL, phi_out [nrhs][N]); they must stay valid until
 *     the problem is removed.  The problem starts from phi = 0 at the next
 *     step.  tol >= 0, 1 <= max_iters < 2^30.  Allocates the workspaces now
 *     (JSWEEP_ERR_OOM if that fails; nothing is added then).
 *   jsweep_batch_step: up to n_sweeps source iterations of every active
 *     problem, then waits for them; a problem that finished during the call
 *     has phi_out written (on the device, by the iteration that finished it)
 *     before the call returns.  *n_active (may be NULL) receives the number
 *     of problems still iterating.
 *   jsweep_batch_launch / jsweep_batch_poll: jsweep_batch_step in two
 *     halves, so that one host thread can keep several batches (each on its
 *     own stream) busy at once: launch queues up to n_sweeps iterations and
 *     returns; poll reports *done = 1 once they have finished (with wait != 0
 *     it waits for them) and then updates the states and *n_active (may be
 *     NULL).  A batch takes one launch at a time; the other batch calls wait
 *     for a pending launch first.
 *   jsweep_batch_query: state (JSWEEP_PROBLEM_*), sweeps done and last
 *     residual of a problem (pointers may be NULL).
 *   jsweep_batch_remove: drops a problem and frees its workspaces.
 *   jsweep_batch_source_iterate: restarts every problem from phi = 0 and
 *     steps until none is active; iters_out / resid_out (host, may be NULL)
 *     receive one entry per problem in increasing id.  Returns
 *     JSWEEP_ERR_NOT_CONVERGED if a problem stopped at max_iters.
 *   jsweep_batch_autotune: for each candidate (cluster_cells, angles_per_warp,
 *     unit_order) times one batched iteration and keeps the fastest; *best_ms
 *     (may be NULL) receives its time.  It restarts every problem from
 *     phi = 0, as jsweep_batch_source_iterate does.
 *   jsweep_batch_options: the batch's current options (after
 *     jsweep_batch_autotune: the chosen ones).
 *   jsweep_batch_stats: device time of the last batched sweep launch and of
 *     the whole last iteration, in ms, the number of kernels the batch has
 *     launched since it was created, and the host time spent (and the number
 *     of times) rebuilding its merged tables and captured iteration after the
 *     problem set changed (pointers may be NULL).
 */
#define JSWEEP_BATCH_MAX_PROBLEMS 65536
#define JSWEEP_PROBLEM_ACTIVE 0    /* still iterating */
#define JSWEEP_PROBLEM_CONVERGED 1 /* residual below tol; phi_out written */
#define JSWEEP_PROBLEM_MAX_ITERS 2 /* stopped at max_iters; phi_out written */
JSWEEP_API int jsweep_batch_create(int precision, int nrhs, const jsweep_options *opt, jsweep_batch_t *out);
JSWEEP_API int jsweep_batch_problem_bytes(jsweep_batch_t batch, jsweep_dags_t dags, int has_inflow,
                                          int64_t *bytes);
JSWEEP_API int jsweep_batch_add(jsweep_batch_t batch, jsweep_dags_t dags, const void *sigma_t,
                                const void *c_ratio, const void *q, const void *inflow, void *phi_out,
                                double tol, int max_iters, int64_t *id, void *stream);
JSWEEP_API int jsweep_batch_step(jsweep_batch_t batch, int n_sweeps, int64_t *n_active, void *stream);
JSWEEP_API int jsweep_batch_launch(jsweep_batch_t batch, int n_sweeps, void *stream);
JSWEEP_API int jsweep_batch_poll(jsweep_batch_t batch, int wait, int *done, int64_t *n_active);
JSWEEP_API int jsweep_batch_query(jsweep_batch_t batch, int64_t id, int *state, int *iters, double *resid);
JSWEEP_API int jsweep_batch_remove(jsweep_batch_t batch, int64_t id);
JSWEEP_API int jsweep_batch_clear(jsweep_batch_t batch);
JSWEEP_API int jsweep_batch_size(jsweep_batch_t batch, int64_t *n_problems);
JSWEEP_API int jsweep_batch_source_iterate(jsweep_batch_t batch, int *iters_out, double *resid_out,
                                           void *stream);
JSWEEP_API int jsweep_batch_autotune(jsweep_batch_t batch, void *stream, double *best_ms);
JSWEEP_API int jsweep_batch_stats(jsweep_batch_t batch, double *sweep_ms, double *iteration_ms,
                                  int64_t *launches, double *setup_ms, int64_t *rebuilds);
JSWEEP_API int jsweep_batch_options(jsweep_batch_t batch, jsweep_options *out);
JSWEEP_API int jsweep_batch_destroy(jsweep_batch_t batch);

/* ---- source iteration that allocates no device memory ----------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory while they run: for example a host application
 * that owns and budgets all of the device's memory through its own runtime, or a
 * latency-critical solve loop where the device-wide synchronisation of
 * cudaMalloc / cudaFree is not acceptable.
 * Same arguments, arithmetic and results as jsweep_source_iterate (level-by-level
 * schedule), but every temporary (psi, sources, lagged values, phi iterates,
 * residual accumulators) lives in one fixed device array of
 * JSWEEP_NOALLOC_SCRATCH_BYTES that the library defines at file scope; every GPU
 * that loads the library holds that array until the process exits.  The call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine) and
 * does not touch the handle's own sweep workspaces or lagged values.
 *   - Problems whose temporaries exceed the array are rejected with
 *     JSWEEP_ERR_INVALID_ARG (the message gives the bytes needed): roughly
 *     directions x cells x padded right-hand sides x element size must stay
 *     below 64 MiB (e.g. 4,096 cells x 96 directions x 1 rhs in FP64 fits).
 *   - The array belongs to the library's device code: the first use of the
 *     library on a device loads that code and commits the array there (64 MiB),
 *     and the first call of this function on a device looks up the array's
 *     address with that device current.  A caller that budgets all of the
 *     device's memory should make one small call (any built handle) before it
 *     takes its budget.
 *   - The function synchronises `stream` at every iteration (it reads the
 *     residual on the host to decide whether to stop), so it cannot be called
 *     while the stream is being captured into a CUDA graph.
 *   - All calls share the one array and it keeps the last call's contents (each
 *     call zeroes what must start at zero), so calls that overlap on the GPU
 *     (different streams or threads) race: serialise them.
 *   - The handle must have been built (jsweep_build_dags); its level arrays,
 *     lag lists, mesh and directions are read, never written. */
#define JSWEEP_NOALLOC_SCRATCH_BYTES (64ull << 20)
JSWEEP_API int jsweep_source_iterate_noalloc(jsweep_dags_t dags, int nrhs, int precision, const void *sigma_t,
                                  const void *c_ratio, const void *q, const void *inflow, double tol,
                                  int max_iters, void *phi_out, int *iters_out, double *resid_out,
                                  void *stream);

/* ---- timing of the last sweep call on a handle (phase breakdown, Sec. VI-C) */
typedef struct {
    double build_ms;        /* last jsweep_build_dags: device time of the whole build */
    double sweep_ms;        /* last sweep kernel(s) only */
    double phi_ms;          /* last phi reduction */
    int64_t sweep_launches; /* kernels launched by the last sweep (graph nodes included) */
    int64_t build_launches; /* kernels launched by the last jsweep_build_dags */
    int64_t call_launches;  /* kernels launched by the last jsweep_sweep / jsweep_source_iterate */
    int64_t build_steps;    /* frontier steps of the last build (about the largest level count) */
    int64_t build_stall_rounds; /* cycle-resolution rounds of the last build, summed over directions */
    double build_phase_ms[6];   /* last build, device time per phase: [0] octant diagonals, [1] set-up and
                                   face classification, [2] frontier steps with cycle resolution,
                                   [3] level-major order, [4] lag lists, [5] schedule layers */
    int64_t sweep_programs; /* JSWEEP_MODE_PATCH: (patch, octant) programs of the last sweep */
    int64_t sweep_requeues; /* JSWEEP_MODE_PATCH: programs the last sweep queued again after a yield */
} jsweep_timing;
JSWEEP_API int jsweep_dags_timing(jsweep_dags_t dags, jsweep_timing *t);

#ifdef __cplusplus
}
#endif
#endif /* JSWEEP_H */
