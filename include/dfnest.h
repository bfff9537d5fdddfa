/*
 * dfnest.h -- C ABI of libdfnest.so, the GB300 (sm_103a) nested-mesh solver of
 * Velasco Romero & Masset (2018), "Numerical study of dynamical friction with
 * thermal effects -- I", Sec. 3 (nested meshes) and Sec. 3.4 (set-up).
 *
 * A context holds one hierarchy of n_levels nested Cartesian meshes, refinement
 * ratio 2 (Sec. 3), all resident in the memory of one GPU.  Level l covers
 * [lo*2^-l, hi*2^-l] with n[0] x n[1] x n[2] active cells and G ghost layers.
 * Fields: 0 rho (density), 1 e (internal energy density), 2..4 v_x, v_y, v_z.
 * rho and e are cell-centred; v_d sits on the lower d-face of its cell (staggered).
 * Host arrays are x-fastest, i.e. index ((k*ny)+j)*nx+i.
 *
 * Conventions shared by every call:
 *  - return value: DF_OK (0) or a negative DF_E* code; df_last_error() gives a
 *    message for the calling thread.  No call aborts the process.
 *  - the context owns every device allocation it makes; the caller owns every
 *    host buffer it passes (read or written synchronously before return).
 *  - work is issued on the stream given at creation (a cudaStream_t, NULL for
 *    the legacy default stream); calls that return host data synchronise it.
 *  - a context is not thread-safe; distinct contexts are independent.
 */
#ifndef DFNEST_H
#define DFNEST_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DF_OK 0
#define DF_EINVAL (-1)     /* bad argument, size or geometry */
#define DF_ENOMEM (-2)     /* device or host allocation failed */
#define DF_ECUDA (-3)      /* a CUDA runtime call failed */
#define DF_EUNHEALTHY (-4) /* NaN, rho <= 0 or e <= 0 found by the time-step reduction */
#define DF_ETIMEOUT (-5)   /* reserved: a bounded device wait ran out */
#define DF_EBUSY (-6)      /* reserved: no capacity */

#define DF_MAX_LEVELS 16

/* level-0 boundary types, one per face -x,+x,-y,+y,-z,+z */
#define DF_BC_PERIODIC 0
#define DF_BC_OUTFLOW 1 /* zero gradient: copy of the nearest active element */
#define DF_BC_INFLOW 2  /* background rho0, e0, V in every ghost element (injection) */
#define DF_BC_REFLECT 3 /* mirror, normal velocity odd (Sec. 3.4 symmetric/antisymmetric) */
/* A reflecting LOWER face at coordinate 0 (lo[d] == 0) is a mirror plane through the
 * perturber: the quadrant domain of Sec. 3.4.  The run then stands for the domain
 * unfolded across the plane.  Every level starts on the plane and takes the reflect
 * fill there.  The luminosity goes to the unfolded domain's cells.  The force is the
 * unfolded one: zero along a mirror axis, 2^planes times the simulated part's sum for
 * the other components. */

/* state precision */
/* DF_FP64: 8 bytes per state value, each value a double with at most 47 significant
 * bits (stored as a float pair hi + lo, which the stencils compute with: double-float
 * arithmetic, 48-bit significands); force, time step, flux sums, CommMean and the
 * boundary fill in FP64.  Values read out (df_get_field, df_get_state) are exact;
 * values written in (df_set_field, df_set_state) are rounded to the 47 bits, and a
 * state read out and written back is restored bit for bit. */
#define DF_FP64 0
#define DF_FP32_STATE 1 /* FP32 state and stencils; FP64 force, time step, flux sums */

typedef struct {
  double gamma;       /* adiabatic index; p = (gamma-1) e (Sec. 2.1) */
  double rho0;        /* background density (Sec. 3.4) */
  double cs;          /* background adiabatic sound speed; e0 = cs^2 rho0/(gamma(gamma-1)) */
  double mach;        /* |V|/cs of the wind */
  double flow_dir[3]; /* unit vector of the wind V (the perturber moves along -V) */
  double GM;          /* perturber mass, Plummer potential Phi = -GM/sqrt(r^2+eps^2) (Eq. 16) */
  double eps;         /* softening length, also in the force sum (Eq. 18) */
  double chi;         /* thermal diffusivity (Eq. 3, Eqs. 19-22) */
  double L;           /* luminosity (Sec. 3.4): L dt added per level step */
  double lum_sigma;   /* 0: split over the 8 cells at the vertex; >0: Gaussian, this sigma */
  double cfl;         /* Courant number of the advective limit */
  double cfl_diff;    /* safety factor of the explicit-diffusion limit 1/(2 chi sum dx^-2) */
  double dt_fixed;    /* >0: coarse step used instead of the reduction */
  int xi_mode;        /* 0: xi = 2 on every level (Sec. 3.1); 1: Eq. 55-56 search per step */
  int bc[6];          /* DF_BC_* of level 0 */
  int diff_face_rho;  /* 0: face density = mean of the two cells (Eq. 3); 1: rho0 (Eqs. 19-21) */
  int hydro_on;       /* 0 freezes rho and v (pure diffusion) */
  int band;           /* CommMean band width in coarse cells (Sec. 3.2.2); default 5 */
  double av_c2;       /* SubStep2 (Sec. 3.3): von Neumann-Richtmyer artificial viscosity
                         coefficient in the ZEUS form (Stone & Norman 1992); 0 = off.
                         With it on, every operator sweeps the whole padded array. */
} df_params;

/* Device memory.  By default the library allocates with cudaMalloc and frees with
 * cudaFree.  df_set_allocator makes every context and pool created afterwards take
 * all its device buffers from alloc(bytes, user), for example PyTorch's caching
 * allocator.  It returns them through dealloc(ptr, user) when the owner is
 * destroyed (or a plan buffer grows).  Each owner keeps the allocator it was
 * created with (a pool's runs: the one current at their admission), so changing
 * it later affects only new owners.  alloc returns NULL on failure, which the
 * creating call reports as DF_ENOMEM.  It must return 256-byte aligned device
 * memory of the current device; a misaligned block is handed back and reported as
 * DF_ECUDA.  (NULL, NULL, NULL) restores cudaMalloc / cudaFree.  alloc and dealloc
 * are set together (DF_EINVAL otherwise).  Not synchronised with concurrent
 * df_create / df_pool_create / df_pool_admit calls. */
typedef void* (*df_alloc_fn)(size_t bytes, void* user);
typedef void (*df_free_fn)(void* ptr, void* user);
int df_set_allocator(df_alloc_fn alloc, df_free_fn dealloc, void* user);

typedef struct df_ctx df_ctx;

/* Create a hierarchy (Sec. 3, Sec. 3.4).  n[d] % 4 == 0, n[d] >= 8, n[d] >= G; G even
 * and >= 2 (G >= 8 makes the active cells independent of the ghost width); every finer level
 * must sit on parent faces with its ghosts and the 27-point CommUp stencil inside
 * the parent's active cells (offset >= G/2+1 parent cells on each side), except on an
 * axis with lo[d] == 0, where every level starts on that face (offset 0, so n[d] >= G+2)
 * and df_set_params then requires bc[2d] == DF_BC_REFLECT (a mirror plane).
 * precision: DF_FP64 or DF_FP32_STATE.  device: CUDA ordinal (made current).
 * stream: cudaStream_t or NULL.  The state is uninitialised until df_set_params.
 * Errors: DF_EINVAL (geometry), DF_ENOMEM, DF_ECUDA. */
int df_create(df_ctx** out, int n_levels, const int n[3], const double lo[3], const double hi[3],
              int G, int precision, int device, void* stream);

/* df_create with a ground level of its own: level 0 has n0[3] cells over [lo, hi],
 * every finer level n[3] cells.  The cell halves from level to level, so level
 * l >= 1 spans [lo, hi] scaled about the origin by (n[d]/n0[d]) 2^-l per axis.
 * n0 = 2n is the hierarchy of Sec. 4.1.1 whose first level covers a quarter of the
 * ground's extent (a 64x64x128 ground under levels of 32x32x64); n0 = n is
 * df_create.  The nesting rules of df_create hold level by level (the ground has
 * its own count in them), and n0 obeys the same size rules as n.  Ownership and
 * errors as df_create. */
int df_create_ground(df_ctx** out, int n_levels, const int n0[3], const int n[3],
                     const double lo[3], const double hi[3], int G, int precision, int device,
                     void* stream);

/* The problem statement's constructor (Sec. 3: n_levels nested meshes, refinement
 * ratio 2, centred on the perturber; Sec. 3.4: the coarse box): N^3 active cells on
 * every level, level l spanning [coarse_lo 2^-l, coarse_hi 2^-l], and
 * DF_DEFAULT_GHOST ghost layers (twice the reach of one level step, so the active
 * cells do not depend on the ghost width).  Equivalent to df_create with
 * n = (N, N, N) and G = DF_DEFAULT_GHOST, except that device memory comes from
 * alloc(bytes, user) / dealloc(ptr, user) when they are given (both or neither;
 * same contract as df_set_allocator: 256-byte aligned memory of `device`, NULL on
 * failure); with both NULL, from the allocator df_set_allocator installed, else
 * cudaMalloc.  The context keeps the callbacks until df_destroy.  Errors as
 * df_create; DF_EINVAL when only one callback is given. */
#define DF_DEFAULT_GHOST 8
int df_create_levels(df_ctx** out, int n_levels, int N, const double coarse_lo[3],
                     const double coarse_hi[3], int precision, int device, void* stream,
                     df_alloc_fn alloc, df_free_fn dealloc, void* user);

/* Copy the parameters, precompute the static potential (Eq. 16) and luminosity
 * weights, and set every level to the uniform background (Sec. 3.4): rho0, e0, V.
 * Resets t to 0 and clears the force history.  DF_EINVAL on bad values, and when
 * finer levels start on a lower face at coordinate 0 that does not reflect. */
int df_set_params(df_ctx* ctx, const df_params* p);

/* Advance n coarse steps: per step the time step of Eq. 55 (reductions on the
 * device), then the recursion of Sec. 3.3 (finer levels first, xi sub-cycles,
 * CommFlux, CommUp, CommMean), then the force of Eq. 18.  With xi_mode = 1 the
 * Eq. 55-56 search also runs on the device each step and the second sub-cycles
 * of levels with xi = 1 do no work, so either mode replays one CUDA graph.
 * t_out NULL: asynchronous on the context's stream, and DF_EUNHEALTHY is reported
 * by the next synchronising call.  t_out given: the call synchronises, writes the
 * simulated time after the steps and returns DF_EUNHEALTHY if the state went bad. */
int df_step(df_ctx* ctx, int n_coarse_steps, double* t_out);

/* Synchronise, then return time, last coarse step and health (0 healthy). */
int df_status(df_ctx* ctx, double* t, double* dt_last, int* unhealthy);

/* Force on the perturber after the last coarse step (Eq. 18 with rho - rho0,
 * covered coarse cells excluded), FP64.  F_along_motion (nullable) = F . (-V/|V|).
 * Synchronises.  Before any step it is the force of the current state. */
int df_force(df_ctx* ctx, double F_out[3], double* F_along_motion);

/* Recompute the force of the current state now (does not advance). */
int df_force_now(df_ctx* ctx, double F_out[3]);

/* Time step the next coarse step would take (Eq. 55) and the per-level limits
 * (dt_level nullable, n_levels entries).  Synchronises. */
int df_compute_dt(df_ctx* ctx, double* dt, double* dt_level);

/* Active cells of one field of one level as FP64 (n0*n1*n2, x fastest). Sync. */
int df_get_field(df_ctx* ctx, int level, int field, double* host_out);
int df_set_field(df_ctx* ctx, int level, int field, const double* host_in);

/* Whole padded array ((n+2G)^3 elements, x fastest) of one field, FP64. Sync. */
int df_get_full(df_ctx* ctx, int level, int field, double* host_out);
int df_set_full(df_ctx* ctx, int level, int field, const double* host_in);

/* Checkpoint: every padded field of every level as stored -- the deviation from
 * the uniform background (rho - rho0, e - e0, v - V), converted to FP64 -- in the
 * order level-major, field-minor, plus the time t; each (level, field) block has
 * the element count of the largest level (a smaller level fills the start of its
 * block).  df_state_size gives the element count.  Restoring a saved state resumes
 * a run bitwise. */
size_t df_state_size(const df_ctx* ctx);
int df_get_state(df_ctx* ctx, double* host_out, double* t_out);
int df_set_state(df_ctx* ctx, const double* host_in, double t);

/* Inter-level operators on demand (Sec. 3.2): CommUp fills every ghost element
 * of level coarse_level+1 from coarse_level; CommMean overwrites the band of
 * coarse_level from coarse_level+1; fill_bc applies the level-0 boundaries. */
int df_prolong(df_ctx* ctx, int coarse_level);
int df_restrict(df_ctx* ctx, int coarse_level);
int df_fill_bc(df_ctx* ctx);

/* Number of kernels launched by this context since creation (counts every
 * launch, graph replays included). */
long long df_kernel_launches(const df_ctx* ctx);

/* Timing hook.  With timing on, df_step launches without the CUDA graph and
 * brackets every kernel with a pooled pair of CUDA events on the context's
 * stream (no host synchronisation inside a step).  df_kernel_time synchronises,
 * then returns the summed device time (ms) and launch count of one kernel kind
 * since df_set_timing; df_kernel_name(kind) names the kinds 0..DF_KERNEL_KINDS-1.
 * df_set_timing resets the totals. */
#define DF_KERNEL_KINDS 18
int df_set_timing(df_ctx* ctx, int on);
int df_kernel_time(df_ctx* ctx, int kind, double* ms, long long* launches);
const char* df_kernel_name(int kind);

/* Tile autotuner: times every operator and sweep direction of one coarse step for
 * each of the library's tile shapes (the order in which a block enumerates the
 * elements of a box: flat, or 256-element (x,y,z) tiles 32x8x1, 32x1x8, 32x4x2,
 * 64x4x1), keeps the fastest, and restores the state, so tuning does not advance
 * the run.  tiles_out (nullable) receives DF_POOL_OPS x 3 shape indices.  The choice
 * changes the order of work only: results are bitwise unchanged. */
int df_autotune(df_ctx* ctx, int* tiles_out);
/* Set the tile shape (0..4, in the order above) of every operator and direction:
 * shapes[3 * op + d].  DF_EINVAL for a null pointer or a shape out of range. */
int df_set_tile_shapes(df_ctx* ctx, const int* shapes);

/* Transport kernels (Sec. 3.1 sweeps).  DF_TRANSPORT_SEPARATE: four kernels per sweep
 * (e/rho and Pi/rho_face; mass and energy fluxes; momentum fluxes; conservative
 * update) exchanging their results through HBM.  DF_TRANSPORT_FUSED: one kernel per
 * sweep that keeps them in shared memory for a tile plus its halo (the halo's
 * quotients and fluxes are recomputed by neighbouring tiles) and ping-pongs the
 * state through a second copy; about a third of the memory traffic.  The two give
 * the same arithmetic on every active cell (equal up to the compiler's contraction
 * of multiply-adds).  DF_TRANSPORT_AUTO (default): separate for DF_FP64 (its
 * kernels are bound by the FP64 pipe); for DF_FP32_STATE fused in pools of several
 * runs and, for a single run, on levels of at least 512 Ki active cells (the sweeps
 * leave one small box short of blocks). */
#define DF_TRANSPORT_AUTO 0
#define DF_TRANSPORT_SEPARATE 1
#define DF_TRANSPORT_FUSED 2
int df_set_transport(df_ctx* ctx, int mode);

/* Verification switch: with on != 0 every operator runs over its whole stencil
 * range in the padded array (the ghost layers evolve exactly as in a plain
 * sweep of the whole array) instead of the active box plus the reach margin.
 * Active cells are identical either way when G >= 8. */
int df_debug_full_boxes(df_ctx* ctx, int on);

int df_destroy(df_ctx* ctx);

/* Self-check of the FP64 division the stencil kernels use (Newton-Raphson on the
 * hardware reciprocal estimate, Markstein 1990) against IEEE division on the current
 * device: n operand pairs from host arrays; *max_ulp receives the largest difference
 * in units in the last place of the IEEE quotient.  Synchronous. */
int df_check_division(const double* a, const double* b, int n, double* max_ulp);

/* Self-check of the double-float arithmetic (a float pair hi + lo, the FP64 state's
 * stencil arithmetic) on the current device: n operand pairs from host arrays;
 * worst[8] (caller-owned, 8 doubles) receives the largest error of conversion from
 * double, sum, product and quotient against FP64, each in units of its bound: 2^-45
 * |a|, 2^-46 (|a| + |b|), 2^-46 |a b| + 2^-120, 2^-42 |a / b| + 2^-120; then of the
 * unnormalised product and quotient the stencils use where a result only feeds more
 * arithmetic (the same two bounds), the size of their low parts against 2^-21 of
 * their high parts, and a sum taking the unnormalised product, against 2^-45 (|a b| +
 * |a|) + 2^-120 (<= 1 passes).  Synchronous. */
int df_check_df64(const double* a, const double* b, int n, double* worst);

/* Measured FP64 throughput of the device: a kernel of independent chains of
 * dependent fused multiply-adds over 8 blocks of 256 threads per SM, timed with CUDA
 * events (best of `repeats` after one warm-up launch).  *tflops receives the FP64
 * flops per second / 1e12 (a multiply-add counts 2), *ms_best (nullable) the best
 * launch's duration.  It is the denominator of the FP64 kernels' ALU roofline.
 * Allocates 8 bytes of device memory for the duration of the call. */
int df_measure_fp64_peak(int device, int repeats, double* tflops, double* ms_best);

/* Force of one level without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- a host whose
 * device memory is entirely reserved by another allocator, a latency-critical loop
 * that cannot afford cudaMalloc's implicit device synchronisation, or a sandboxed
 * plug-in that is not allowed to allocate.  It sums, over the active cells of one
 * level whose centre lies outside the covered box, GM times (rho - rho0) times the
 * cell volume times r / (r^2 + eps^2)^(3/2), r the cell centre's position relative
 * to the perturber at the origin -- the same per-level sum as the context's force
 * reduction.  Its scratch -- one triple of partial sums per 256 active cells -- is a
 * fixed file-scope device array of DF_NOALLOC_MAX_CELLS/256 triples (384 KiB) that
 * every GPU loading the library holds until the process exits.
 *  rho: device pointer to the padded FULL density of the level ((n+2G)^3, x fastest),
 *    as df_get_full returns it -- not the deviation rho - rho0 a context stores;
 *  n, G, lo (lower corner of the active box), dx: the level's geometry (host arrays);
 *  child_off, child_n: the covered box in this level's active cells (offset and
 *    extent, the child's cell counts halved; 0 <= child_off[d], 1 <= child_n[d],
 *    child_off[d] + child_n[d] <= n[d]), both NULL for a level without a child;
 *  GM, eps, rho0: perturber mass, softening length, background density;
 *  mirror: bit d set when the lower face of axis d is a mirror plane through the
 *    perturber (a quadrant-domain context): the result is then the unfolded domain's,
 *    as df_force_now gives it -- 0 along each mirror axis, 2^(bits set) times the
 *    simulated part's sum for the others; 0 for a whole-domain level;
 *  F_out: device pointer to 3 doubles (written).
 * The first call on a device looks up the array's device address once (with that
 * device current); make that first call before any stream capture.  Every call uses
 * the same array and leaves its contents behind; each call writes every partial it
 * reads, so nothing needs clearing, but calls whose work overlaps on the GPU (on
 * different streams, or from several threads) race on the array and give wrong sums.
 * Asynchronous on `stream`.  DF_EINVAL for null pointers, bad sizes, a covered box
 * outside the level, a mirror mask outside 0..7 or more than DF_NOALLOC_MAX_CELLS
 * active cells; DF_ECUDA if the lookup or a launch fails.  It calls no cudaMalloc,
 * cudaFree or allocating library routine. */
#define DF_NOALLOC_MAX_CELLS 4194304
int df_force_level_noalloc(const double* rho, const int n[3], int G, const double lo[3],
                           const double dx[3], const int child_off[3], const int child_n[3],
                           double GM, double eps, double rho0, int mirror, double* F_out,
                           void* stream);

/* ---- Batched runs (pools).  A pool holds many independent hierarchies ("runs",
 * e.g. a parameter sweep or a stream of simulation requests) on one GPU and
 * advances all of them together: one coarse step of every run is one sequence of
 * persistent work-list launches, each carrying the same operator (Sec. 3.3 level
 * step, CommUp, CommMean, Eq. 55 and Eq. 18 reductions) for every run that has it
 * next, captured once into a CUDA graph.  Runs may differ in level count, mesh
 * size and physics; every run sub-cycles with xi = 2 and takes its own time step. */
typedef struct df_pool df_pool;

/* Device bytes one run of this shape holds (the pool's admission measure). */
size_t df_run_bytes(int n_levels, const int n[3], int G, int precision);
/* The same for a run with a ground level of n0[3] cells (df_create_ground). */
size_t df_run_bytes_ground(int n_levels, const int n0[3], const int n[3], int G, int precision);

/* Create an empty pool that admits runs while their bytes stay within
 * hbm_budget_bytes.  precision as in df_create (one precision per pool). */
int df_pool_create(df_pool** out, size_t hbm_budget_bytes, int precision, int device,
                   void* stream);

/* Admit one run (arguments as df_create + df_set_params); returns its slot.
 * DF_EBUSY when the budget would be exceeded (nothing is allocated then);
 * DF_EINVAL for bad shapes or parameters.  Runs with xi_mode = 1 choose their
 * sub-cycling on the device each coarse step, as in a context. */
int df_pool_admit(df_pool* pool, int n_levels, const int n[3], const double lo[3],
                  const double hi[3], int G, const df_params* p, int* slot_out);
/* Admit a run with a ground level of n0[3] cells (geometry as df_create_ground). */
int df_pool_admit_ground(df_pool* pool, int n_levels, const int n0[3], const int n[3],
                         const double lo[3], const double hi[3], int G, const df_params* p,
                         int* slot_out);

/* Free a run's slot and memory (synchronises the pool's stream first). */
int df_pool_release(df_pool* pool, int slot);

/* Advance every admitted run by n coarse steps (asynchronous). */
int df_pool_step(df_pool* pool, int n_coarse_steps);

/* Synchronise, then write 6 doubles per slot (slots 0..max_slots-1): F_x, F_y,
 * F_z of the last coarse step, t, the last coarse dt, and the health flag (NaN for
 * empty slots).  Returns the number of slots written. */
int df_pool_query(df_pool* pool, double* out, int max_slots);

/* Force on the perturber of one slot's run after its last coarse step (Eq. 18, as
 * df_force) and its simulated time (t_out nullable).  Synchronises the pool's
 * stream.  DF_EINVAL for an empty slot; DF_EUNHEALTHY (outputs still written) when
 * that run's state went bad -- the other slots are unaffected. */
int df_pool_force(df_pool* pool, int slot, double F_out[3], double* t_out);

/* Force history of one slot's run: the last min(k, steps taken, 4096) coarse steps,
 * oldest first, 4 doubles each -- F_x, F_y, F_z after the step (Eq. 18) and the time
 * at its end -- written to out (4k doubles); *got receives the entry count.
 * Synchronises the pool's stream.  A server can step a run several coarse steps
 * between two reads and still test a convergence rule at every step.  DF_EINVAL for
 * an empty slot, a null pointer or k < 0. */
int df_pool_history(df_pool* pool, int slot, int k, double* out, int* got);

/* Active cells of one field of one level of a slot's run, FP64 (as df_get_field). */
int df_pool_get_field(df_pool* pool, int slot, int level, int field, double* host_out);
/* Set the active cells of one field of one level of a slot's run (as df_set_field). */
int df_pool_set_field(df_pool* pool, int slot, int level, int field, const double* host_in);

/* Active runs, bytes in use, the budget, kernels launched so far. */
int df_pool_info(df_pool* pool, int* active, size_t* used, size_t* budget, long long* launches);

/* Tile and grid shape of the work-list launches.  df_pool_set_tiles sets the
 * persistent blocks per SM of each of the DF_POOL_OPS operators.  df_pool_autotune
 * times every operator of one coarse step of the current runs for 1..32 blocks per
 * SM and for each tile shape (as df_autotune), keeps the fastest per operator
 * (blocks per SM written to blocks_per_sm_out, nullable) and restores the runs'
 * state. */
#define DF_POOL_OPS 22
int df_pool_set_tiles(df_pool* pool, const int* blocks_per_sm);
int df_pool_autotune(df_pool* pool, int* blocks_per_sm_out);
/* As df_set_transport, for every run of the pool. */
int df_pool_set_transport(df_pool* pool, int mode);
/* As df_set_tile_shapes, for every run of the pool. */
int df_pool_set_tile_shapes(df_pool* pool, const int* shapes);

/* Timing hook of a pool (as df_set_timing / df_kernel_time). */
int df_pool_set_timing(df_pool* pool, int on);
int df_pool_kernel_time(df_pool* pool, int kind, double* ms, long long* launches);

int df_pool_destroy(df_pool* pool);

/* Eq. 55-56 (Appendix A): brute force over xi in {1,2}^(n-1), maximising dt/C. */
int df_xi_search(int n, const double* dt_level, const double* cost, int* xi_out, double* ratio);

/* Message of the last error on the calling thread ("" if none). */
const char* df_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
