/*
 * hot_mpm.h -- C ABI of the GB300 (sm_103a) implementation of the implicit
 * MPM time step "Hierarchical Optimization Time Integration" (HOT), Wang et
 * al., arXiv 1911.07913.
 *
 * One call sequence advances one scene by one implicit-Euler step, following
 * the operation sequence of Sec. 3.1 (P2G, grid time step, G2P, strain
 * update, advection):
 *
 *     mpm_p2g(s);            bin/sort particles, APIC P2G, boundary conditions
 *     mpm_solve_step(s, &st) minimise Eq. 1 with HOT (Alg. 3, V-cycle Alg. 2), or
 *                            with the paper's comparison solvers (Alg. 1) by option
 *     mpm_g2p(s);            APIC G2P, F update, advection
 *
 * or mpm_step() for the three.  All arithmetic runs in the library's CUDA
 * kernels on the stream given at creation; there is no CPU fallback.
 *
 * Conventions
 *   - Every function returns an mpm_status; nothing throws across the ABI.
 *     mpm_last_error(s) returns a message for the last failure on s
 *     (thread-local when s is NULL).
 *   - Particle arrays are row-major AoS as a caller holds them: x, v (n x 3),
 *     F, C (n x 3 x 3, F[p*9 + 3a + b] = F_ab), vol, mass (n), all float64;
 *     material_id (n) int32.  "host" or "device" as the flag says.
 *   - Grid nodes are integer triples (i, j, k), node position origin + dx*(i,j,k);
 *     a scene's active nodes are the union of its particles' 3x3x3 quadratic
 *     B-spline stencils, listed in (k, j, i)-lexicographic order.
 *   - Node vectors (dv, g, b, u) are n_nodes x 3 float64, row-major.
 *   - The library owns every device buffer it allocates; caller pointers are
 *     only read or written during the call.
 *   - Calls on one scene are not thread-safe; different scenes are
 *     independent.
 */
#ifndef HOT_MPM_H
#define HOT_MPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_scene *mpm_scene_t;

typedef enum {
  MPM_OK = 0,
  MPM_ERR_INVALID_ARG = 1,   /* null pointer, bad size or option */
  MPM_ERR_OOM = 2,           /* device allocation failed */
  MPM_ERR_CUDA = 3,          /* a CUDA call failed (message has the code) */
  MPM_ERR_NOT_CONVERGED = 4, /* iteration cap reached; state = last accepted iterate */
  MPM_ERR_LINESEARCH = 5,    /* no energy decrease within max_ls halvings */
  MPM_ERR_NUMERIC = 6,       /* NaN/Inf in a norm or energy */
  MPM_ERR_ADMISSION = 7,     /* serving: footprint exceeds the memory budget */
  MPM_ERR_STATE = 8,         /* call out of order (p2g -> solve -> g2p) */
  MPM_ERR_DOMAIN = 9,        /* a particle stencil leaves the grid */
  MPM_ERR_TIMEOUT = 10       /* a bounded device-side wait gave up */
} mpm_status;

/* Material (Sec. 6.1, Table 2).  model 0: fixed corotated (Stomakhin et al.
 * 2012); 1: compressible Neo-Hookean.  plasticity, applied once per step
 * after the F update (lagged, Sec. 2.2): 0 none; 1 von Mises, the
 * deviatoric principal Hencky strain returned onto 2 mu |dev ln s| =
 * yield_stress (yield_stress > 0 required); 2 snow-like clamp of the
 * singular values of F into [0.99, 1.001] (Table 2). */
typedef struct {
  double E, nu, rho, yield_stress;
  int32_t model;
  int32_t plasticity;
} mpm_material;

/* Dirichlet box (Sec. 4.1: boundary conditions by projection).  A node whose
 * position lies in [lo, hi] (inclusive, per axis) is held: type 0 prescribes
 * v = 0, type 1 prescribes v = omega * axis x (x_i - center).  With
 * radius > 0 the region is the box intersected with the cylinder of that
 * radius about the line through center along axis (axis a unit vector): a
 * region the prescribed rotation maps onto itself, so material that starts
 * inside stays inside as it turns.  Boxes apply in list order.
 * Independently of the list, nodes within 3 cells of the grid walls are
 * held at v = 0. */
typedef struct {
  int32_t type;
  int32_t reserved;
  double lo[3], hi[3], axis[3], center[3];
  double omega;
  double radius;
} mpm_bc;

typedef struct {
  int64_t n_particles;
  const double *x, *v, *F, *C, *vol, *mass; /* see layout above; C may be NULL (= 0) */
  const int32_t *material_id;               /* may be NULL (= material 0) */
  const mpm_material *materials;            /* host array */
  int32_t n_materials;
  int32_t grid_dims[3];                     /* cells per axis; nodes 0..grid_dims */
  double dx;
  double origin[3];
  double gravity[3];
  const mpm_bc *bcs;                        /* host array, may be NULL */
  int32_t n_bcs;
  int32_t inputs_on_device;                 /* 1: particle arrays are device pointers */
  void *cuda_stream;                        /* cudaStream_t, NULL = legacy default stream */
} mpm_scene_desc;

/* Solver options; the paper's settings (Sec. 6.1) are eps = 1e-7, cn_mode 0,
 * lbfgs_m = 8, levels = 3, cfl = 0.6, fps = 24. */
typedef struct {
  double eps;            /* termination tolerance */
  int32_t cn_mode;       /* 0: ||g^||_2 <= eps sqrt(n) with the node-wise CN
                            of Sec. 5.2;  1: ||g||_2 <= eps ||g^1||_2 */
  int32_t lbfgs_m;       /* L-BFGS window w (1..16) */
  int32_t levels;        /* multigrid levels M (1..8) */
  int32_t precision;     /* 0: FP64 everywhere; 1: FP32 Hessian, smoother and
                            coarse solve, FP64 energy/gradient/L-BFGS/CN */
  int32_t max_iters;     /* L-BFGS iteration cap */
  int32_t max_ls;        /* line-search halvings cap */
  int32_t max_coarse_cg; /* coarsest-level PCG cap; 0 = number of coarse DOFs, at most 200 when
                            the V-cycle runs in FP32 (precision 1; the coarsest PCG then computes
                            in FP64 on the FP32 matrix) */
  int32_t record_trace;  /* 1: keep the decision trace (mpm_get_trace) */
  double dt;             /* > 0: fixed step; else min(1/fps, cfl dx / v_max) */
  double fps;
  double cfl;
  int32_t flags;         /* bit 0: run the V-cycle eagerly instead of as a CUDA graph;
                            bit 1: coarsest solve by the cooperative kernel, not the cluster one;
                            bit 2: one launch per Gauss-Seidel color on every level;
                            bit 3: one launch per color on the finest level only (by default
                            each symmetric sweep of each level is one cooperative launch, or
                            one 16-CTA cluster launch (bits 10 and 11) on levels with at most
                            160 (FP64) or 256 (FP32) rows per color whose u fits in shared
                            memory, 64 otherwise);
                            bit 6: cooperative launches on those levels too (bits 2, 3 and 6
                            change launch boundaries only, not the arithmetic);
                            bit 7: residual from half of the symmetric matrix (prefix blocks and
                            the transposed half by atomics; measured slower, an option only);
                            bits 8-9: rows (warps) per block of the one-launch-per-color sweeps:
                            0 -> 8, 1 -> 2, 2 -> 4, 3 -> 16 (launch shape only);
                            bit 10: cluster-launched sweeps read and write u in global memory
                            (by default each CTA of the cluster holds the level's u in shared
                            memory and writes new values into every CTA's copy; same results);
                            bit 11: with u in shared memory, a hardware cluster barrier between
                            colors (by default each CTA waits on its own mbarrier for the bytes
                            of the color's rows, sent by remote stores that count them; same
                            results);
                            bit 4: drive the L-BFGS iterations from the host;
                            bit 5: run them as one CUDA graph whose conditional nodes take every
                            decision on the device (by default the graph is used once the
                            scene's previous solve took 8 or more iterations: building it costs
                            about as much as a few host-driven iterations; profiling and bit 0
                            select the host loop) */
  int32_t solver;        /* 0: HOT (Alg. 3); the paper's comparison solvers, Alg. 1 inexact
                            projected Newton with the Sec. 5.3 criterion and the Hessian
                            rebuilt at every Newton iterate: 1: PN-PCG (Jacobi-preconditioned
                            CG), 2: PN-MGPCG (CG preconditioned by one V-cycle of a hierarchy
                            rebuilt every Newton iteration, Sec. 4.3).  For 1 and 2, max_iters
                            caps the Newton iterations and each CG run is capped at
                            MPM_PN_MAX_CG iterations. */
  int32_t refresh_every; /* HOT only; an extension, 0 = Alg. 3 as printed (the hierarchy is
                            built once per step): every refresh_every iterations without
                            convergence, rebuild the projected Hessian and its hierarchy at
                            the current iterate and restart the L-BFGS history (in the
                            device-driven loop too, as a conditional graph node). */
  int32_t fallback_after; /* HOT only; an extension, 0 = off: a step that has not converged
                             after fallback_after L-BFGS iterations continues as PN-MGPCG
                             (Alg. 1) from the current iterate, within the same max_iters.
                             Runs the host-driven loop. */
} mpm_solver_opts;

#define MPM_PN_MAX_CG 10000

typedef struct {
  int32_t iters;           /* L-BFGS iterations (Alg. 3 loop trips); Newton iterations for the
                              projected-Newton solvers */
  int32_t ls_trials;       /* energy evaluations in line searches */
  int32_t coarse_cg_iters; /* coarsest PCG iterations over all V-cycles */
  int32_t vcycles;
  double final_norm;       /* the termination norm at exit */
  double energy;           /* E(dv) at exit, Eq. 1 without constants */
  double dt_used;
  int64_t n_particles;
  int64_t n_nodes[8];      /* active nodes per multigrid level */
  int64_t nnz_blocks[8];   /* 3x3 blocks per level */
  int32_t n_levels;
  int32_t status;
  int32_t graph_vcycles;   /* V-cycles run from a captured CUDA graph */
  int32_t device_loop;     /* 1: the L-BFGS iterations ran as one CUDA graph with device-side
                              decisions (conditional nodes); 0: host-driven loop */
} mpm_step_stats;

/* Device memory hook.  alloc(bytes, stream, ctx) returns device memory or
 * NULL; free(ptr, stream, ctx).  Default: cudaMalloc / cudaFree.  The Python
 * binding installs PyTorch's caching allocator.  Set before creating scenes. */
typedef void *(*mpm_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*mpm_free_fn)(void *ptr, void *stream, void *ctx);
mpm_status mpm_set_allocator(mpm_alloc_fn alloc, mpm_free_fn free_fn, void *ctx);

/* Create a scene: copies particles and settings into library-owned device
 * memory.  Errors: INVALID_ARG (null/size/option), OOM, CUDA. */
mpm_status mpm_create_scene(const mpm_scene_desc *desc, const mpm_solver_opts *opts,
                            mpm_scene_t *out);
mpm_status mpm_destroy_scene(mpm_scene_t s);
const char *mpm_last_error(mpm_scene_t s);

/* Replace the options of an existing scene (same constraints as create). */
mpm_status mpm_set_options(mpm_scene_t s, const mpm_solver_opts *opts);

/* Sec. 3.1 P2G: sort particles by cell (bit-exact cell keys), build the
 * active node set, APIC transfer of mass and momentum, mass-weighted xi_i
 * for the characteristic norm (Sec. 5.2), Dirichlet nodes, and the step size
 * dt.  Errors: DOMAIN when a stencil leaves the grid. */
mpm_status mpm_p2g(mpm_scene_t s);

/* Projected Hessian at dv = 0 (Alg. 3 "projectHessian") and the Galerkin
 * hierarchy H^{m+1} = R H^m P (Eq. "buildMultigrid").  mpm_solve_step calls
 * it when needed; exposed for inspection.  Requires mpm_p2g. */
mpm_status mpm_build_hierarchy(mpm_scene_t s);

/* Alg. 3: minimise Eq. 1 over dv with L-BFGS (window w), the V-cycle of
 * Alg. 2 as initial inverse Hessian, backtracking line search and the
 * termination test of cn_mode.  The grid velocity v^{n+1} = v^n + dv stays on
 * the device.  stats may be NULL.  Errors: NOT_CONVERGED, LINESEARCH,
 * NUMERIC, TIMEOUT; the state then holds the last accepted iterate. */
mpm_status mpm_solve_step(mpm_scene_t s, mpm_step_stats *stats);

/* Sec. 3.1 G2P: APIC velocity and affine matrix, F_p <- (I + dt grad v) F_p,
 * x_p <- x_p + dt v_p.  Requires a solved step. */
mpm_status mpm_g2p(mpm_scene_t s);

/* p2g + solve_step + g2p. */
mpm_status mpm_step(mpm_scene_t s, mpm_step_stats *stats);

/* Particle state in the caller's original order (any pointer may be NULL).
 * to_device: 1 if the pointers are device memory. */
mpm_status mpm_get_state(mpm_scene_t s, double *x, double *v, double *F, double *C,
                         int32_t to_device);
/* Overwrite the particle state (original order; NULL keeps a field). */
mpm_status mpm_set_state(mpm_scene_t s, const double *x, const double *v, const double *F,
                         const double *C, int32_t from_device);

/* Grid after P2G (host pointers, any may be NULL; call with all NULL to get
 * n_nodes): node_ijk (n x 3 int32), m (n), v (n x 3, v^n with prescribed
 * values at held nodes), xi (n), fixed (n, 0/1), dv (n x 3, the last
 * solution, zero before a solve). */
mpm_status mpm_get_grid(mpm_scene_t s, int64_t *n_nodes, int32_t *node_ijk, double *m,
                        double *v, double *xi, int32_t *fixed, double *dv);

/* Eq. 1 energy and its gradient at a caller-given dv (host n x 3), using the
 * current P2G state and dt.  Sec. 3.1 / Sec. 4.1. */
mpm_status mpm_eval_energy(mpm_scene_t s, const double *dv, double *energy);
mpm_status mpm_eval_gradient(mpm_scene_t s, const double *dv, double *grad);

/* Level `level` of the hierarchy as block-CSR (host pointers; call with
 * row_ptr == NULL to get sizes).  cols are node indices of that level,
 * vals are 9 values per block, row-major 3x3, in the precision of the
 * hierarchy converted to float64; coords (n x 3) the level's node triples. */
mpm_status mpm_get_hessian(mpm_scene_t s, int32_t level, int64_t *n_rows, int64_t *nnz_blocks,
                           int32_t *row_ptr, int32_t *cols, double *vals, int32_t *coords);

/* One V-cycle (Alg. 2) applied to b (host n x 3) -> u; cg_iters gets the
 * coarsest PCG count (may be NULL).  Held DOFs of b are ignored, of u zero. */
mpm_status mpm_apply_vcycle(mpm_scene_t s, const double *b, double *u, int32_t *cg_iters);

/* Poll limit of the scene's device-side waits: the grid barrier between the
 * colors of a cooperative Gauss-Seidel sweep and the cooperative coarsest
 * PCG's barriers.  A wait that polls `polls` times without the other blocks
 * arriving gives up: the kernel records the timeout and returns, and the call
 * that launched it returns MPM_ERR_TIMEOUT (its numeric result is then
 * meaningless; the scene stays usable).  Default 2^24 polls (seconds); the
 * paper has no counterpart: this bounds every wait so that a failure cannot
 * hang the GPU, and a small limit lets a test exercise that path.  Errors:
 * INVALID_ARG (polls < 1). */
mpm_status mpm_set_wait_limit(mpm_scene_t s, int64_t polls);

/* Decision trace of the last solve (record_trace = 1): iteration count,
 * accepted step lengths, line-search trials, skipped L-BFGS pairs and
 * restarts per iteration, coarse PCG counts per V-cycle.  Arrays of
 * `capacity` entries; *n_iters and *n_vcycles get the counts. */
mpm_status mpm_get_trace(mpm_scene_t s, int32_t capacity, int32_t *n_iters, double *alphas,
                         int32_t *ls_trials, int32_t *skipped, int32_t *fallback,
                         int32_t *n_vcycles, int32_t *cg_counts);

/* Projected-Newton solvers (solver = 1, 2): CG iterations of each Newton
 * iteration of the last solve.  *n receives the Newton iteration count
 * (entries beyond capacity are not written). */
mpm_status mpm_get_inner_iters(mpm_scene_t s, int32_t capacity, int32_t *n, int32_t *cg_iters);

/* Per-kernel device timing.  mpm_profile(s, 1, only) clears and starts
 * recording CUDA events on the scene's stream around the library's main
 * kernels (only the kernels named in `only`, a comma-separated list, when it is not NULL);
 * mpm_profile(s, 0, NULL) stops.  mpm_profile_read returns, per kernel name (32
 * bytes each in `names`), the summed event time in ms and the launch count;
 * *count gets the number of names (entries beyond capacity are dropped). */
mpm_status mpm_profile(mpm_scene_t s, int32_t enable, const char *only);
mpm_status mpm_profile_read(mpm_scene_t s, int32_t capacity, int32_t *count, char *names, double *total_ms,
                            int64_t *launches);

/* Number of kernels this library has launched in the process so far. */
int64_t mpm_kernel_launch_count(void);

/* Device bytes held by the scene (its admission footprint). */
mpm_status mpm_scene_footprint(mpm_scene_t s, int64_t *bytes);

/* Batched stepping: p2g, solve and g2p of n independent scenes, taken from
 * a shared queue by one worker thread per host core (at most n), the scenes
 * whose previous step in this call took longest first.  Scenes on
 * different streams overlap on the GPU; scenes that share a stream are
 * serialised by it.  stats may be NULL, else n entries (in the order of
 * `scenes`).  Returns the first failing scene's status (mpm_last_error(NULL)
 * names the scene). */
mpm_status mpm_step_batch(mpm_scene_t *scenes, int32_t n, mpm_step_stats *stats);

/* Launch-configuration autotuner for batched stepping (configuration 4 of the
 * benchmark set: many small scenes whose kernels should overlap).  Runs
 * `steps` real batched steps under each candidate -- the V-cycle as a CUDA
 * graph with one cooperative launch per smoothing sweep (options bits 0 and
 * 2 clear), the V-cycle launched eagerly (bit 0), eagerly with one launch
 * per Gauss-Seidel color on every level (bits 0 and 2) or on the finest
 * level only (bits 0 and 3), each with 2, 4, 8 or 16 rows per block of
 * those launches (bits 8-9) -- with half, all and twice the host cores as
 * worker threads, then keeps the fastest: the scenes' bits 0, 2, 3, 8 and 9
 * are set to it and mpm_step_batch uses its worker count from then on.  The
 * candidates differ in launch shape only, so the tuning steps are ordinary
 * steps of the scenes (steps x 10 x the number of distinct worker counts).
 * Outputs (may be NULL): the chosen bits, workers, particle-steps/s and the
 * number of steps each scene took while tuning. */
mpm_status mpm_batch_autotune(mpm_scene_t *scenes, int32_t n, int32_t steps, int32_t *flags_out,
                              int32_t *workers_out, double *rate_out, int32_t *steps_run_out);

/* Residency of a scene's device memory.  park: copy the particle state
 * (positions, velocities, F, C, volumes, masses, material and original ids)
 * to host memory and release every device buffer of the scene (grid,
 * hierarchy and solver storage are rebuilt by the next step, as Alg. 3 builds
 * them per step anyway).  unpark: allocate and copy it back; mpm_p2g,
 * mpm_step, mpm_get_state and mpm_set_state unpark a parked scene by
 * themselves.  residency: *parked (0/1) and *peak_bytes, the largest device
 * footprint the scene has had (what it needs when brought back).  The paper
 * has no counterpart (serving many scenes).  Errors: INVALID_ARG, OOM, CUDA. */
mpm_status mpm_scene_park(mpm_scene_t s);
mpm_status mpm_scene_unpark(mpm_scene_t s);
mpm_status mpm_scene_residency(mpm_scene_t s, int32_t *parked, int64_t *peak_bytes);

/* Continuous-batching step server (serving many scenes) with residency
 * admission.  Requests (one implicit step of a scene each) queue in FIFO
 * order.  The server manages the device memory of every scene submitted to
 * it: the summed footprint of its resident scenes stays within budget_bytes.
 * A request is admitted when a worker is free, its scene is not already
 * being stepped, and room can be made for it: a parked scene needs its peak
 * footprint, a resident one the growth back to its peak; to make room, idle
 * resident scenes are parked, least recently stepped first.  A request for
 * which no room can be made waits while other work is in flight; a lone
 * request is always admitted (so an over-budget mix cannot stall the queue).
 * A scene's first step may overshoot (its peak is unknown before it).  Each
 * worker thread steps its scene with mpm_step on the scene's own stream, so
 * admitted requests overlap on the GPU; create scenes with cuda_stream = NULL
 * so that each gets its own stream, and do not use a scene elsewhere while
 * the server manages it.
 *   submit: MPM_ERR_ADMISSION if the scene alone exceeds the budget.
 *   poll:   *request_id = -1 when nothing has finished (wait = 0) or nothing
 *           is pending (wait = 1); latency = submit -> finish, queue = submit
 *           -> start, seconds; step_status = the step's mpm_status.
 *   destroy: waits for queued and running requests. */
typedef struct mpm_server *mpm_server_t;
mpm_status mpm_server_create(int64_t budget_bytes, int32_t n_workers, mpm_server_t *out);
mpm_status mpm_server_submit(mpm_server_t server, mpm_scene_t scene, int64_t request_id);
mpm_status mpm_server_poll(mpm_server_t server, int32_t wait, int64_t *request_id, mpm_step_stats *stats,
                           double *latency_s, double *queue_s, int32_t *step_status);
mpm_status mpm_server_info(mpm_server_t server, int64_t *queued, int64_t *in_flight, int64_t *in_flight_bytes,
                           int64_t *peak_in_flight_bytes);
/* resident bytes of the managed scenes now and at their peak (sampled after
 * each request), scenes parked and brought back so far, and requests that
 * had to wait for device memory. */
mpm_status mpm_server_residency(mpm_server_t server, int64_t *resident_bytes, int64_t *peak_resident_bytes,
                                int64_t *parks, int64_t *unparks, int64_t *deferred);
mpm_status mpm_server_destroy(mpm_server_t server);

/* FP64 FMA throughput of the current device in TFLOP/s (2 flop per FMA),
 * measured by timing a kernel of independent FMA chains on cuda_stream
 * (NULL = legacy default stream); the best of three timed launches.  The
 * paper has no counterpart: it is the denominator of the FP64-bound kernels'
 * roofline.  Allocates one small scratch buffer.  Errors: INVALID_ARG, OOM,
 * CUDA. */
mpm_status mpm_probe_fp64_fma(void *cuda_stream, double *tflops);

/* Elastic energy sum_p V_p psi(F_p) of a particle set, computed without any
 * device allocation.  The paper has no counterpart: this serves callers that
 * cannot allocate at the point of the call -- real-time loops that cannot
 * afford the device synchronisation cudaMalloc/cudaFree imply, hosts whose
 * device memory is a fixed budget reserved up front by their own pool, and
 * code paths that may not enter an allocator at all.  Every other entry
 * point allocates through the allocator hook.
 *
 * F (n x 9 row-major), vol (n) and material_id (n, may be NULL = material 0;
 * an id outside [0, n_materials) makes the result NaN) are device pointers; materials is a host array of 1..16 entries (models 0
 * and 1 as in mpm_material).  energy receives the sum: a device pointer when
 * energy_on_device is 1 (the call then returns without synchronising),
 * otherwise a host pointer (the call synchronises the stream).
 *
 * Scratch: a fixed 512 KiB array in the library's device memory, held on
 * every GPU that loads the library until the process exits.  Hence the
 * limit n_particles <= 134,217,728 (2048 particles per partial sum); larger
 * sets are rejected with MPM_ERR_INVALID_ARG.  The first call in a CUDA
 * context (per device, and again after a cudaDeviceReset) looks the array's
 * address up (cudaGetSymbolAddress, with that device current); make that
 * first call before any stream capture.  All calls share
 * the array: calls whose work overlaps on the GPU (different streams, or
 * other threads) race and must be serialised by the caller.  Errors:
 * INVALID_ARG, CUDA; message in mpm_last_error(NULL). */
mpm_status mpm_particle_energy_noalloc(const double *F, const double *vol, const int32_t *material_id,
                                       const mpm_material *materials, int32_t n_materials,
                                       int64_t n_particles, double *energy, int32_t energy_on_device,
                                       void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* HOT_MPM_H */
