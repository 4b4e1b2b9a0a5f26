/* UGKWP-LTS steady-iteration step on one B300 GPU: C ABI of libugkwp.so.
 *
 * One step (ugkwp_step) runs, in hand-written sm_103a CUDA kernels on the context's stream:
 *   decomposition W = W^h + W^p and the collisionless fraction e^{-dt_i/tau_i}    (Sec. III B, Sec. IV B)
 *   re-sampling of the hydrodynamic part as new particles                          (Eqs. 25-26, Sec. IV B)
 *   free-flight times t_f = min(-tau_i ln eps, dt_i)                                (Eq. 27, Sec. IV B)
 *   free transport; at every face crossing L -> R the particle mass and its remaining free-transport time
 *     are multiplied by dt_R / dt_L                                                (Eqs. 28, 41, 52)
 *   before/after particle tallies W^{fr,p} = W^{p,+} - W^{p,-}, removal of collided particles (Eqs. 29-30)
 *   time-averaged equilibrium and free-transport wave fluxes with side-normalised coefficients
 *                                                                                   (Eqs. 16, 17-22, 47-50)
 *   the conservative update W^{n+1} = W^n - dt_i/Omega_i sum_j F_j s_j + W^{fr,p}  (Eq. 53)
 *   wall pressure, shear stress and heat flux                                       (Sec. V A)
 * Local time steps come from the CFL condition on the initial freestream field and stay fixed (Eqs. 33-34);
 * GTS mode gives every cell the global minimum.
 *
 * Conventions.
 *  - Every function returns ugkwp_status (0 = OK). ugkwp_last_error gives a message for the last failure.
 *  - The context owns all device memory. Host pointers passed in are owned by the caller and only read or
 *    written during the call.
 *  - ugkwp_step is asynchronous on the context's stream; calls that return host data synchronise it and
 *    report any sticky device-side error (crossing cap, non-physical state, tally overflow). After such an
 *    error the context can only be inspected or destroyed.
 *  - A context is not thread-safe. Units: rho_inf = T_inf = 1, R = 1/2, lengths in the mesh's units.
 *  - Particle order inside a cell after a step is unspecified; the particle set, all integer tallies and
 *    all cell states are deterministic for a given seed.
 */
#ifndef UGKWP_H
#define UGKWP_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct ugkwp_ctx ugkwp_ctx;

typedef enum {
    UGKWP_OK = 0,
    UGKWP_EINVAL = 1,     /* bad argument or mesh */
    UGKWP_ENOMEM = 2,     /* device allocation failed */
    UGKWP_ECUDA = 3,      /* CUDA runtime error */
    UGKWP_ELIMIT = 4,     /* crossing cap (256 per particle per step), particle capacity, > 2047 new / cell */
    UGKWP_ENONPHYS = 5,   /* a non-finite cell state after the update */
    UGKWP_EOVERFLOW = 6   /* a fixed-point tally contribution beyond 2^62 */
} ugkwp_status;

typedef enum { UGKWP_LTS = 0, UGKWP_GTS = 1 } ugkwp_tstep;

/* boundary tags of the mesh's boundary faces */
enum { UGKWP_BC_WALL = 1,      /* diffuse isothermal wall at T_w */
       UGKWP_BC_FARFIELD = 2,  /* freestream ghost on inflow, zero-gradient ghost on outflow; particles leave */
       UGKWP_BC_FIXED = 3,     /* ghost at opts.ghost_state; particles leave */
       UGKWP_BC_SYMMETRY = 4,  /* specular mirror */
       UGKWP_BC_PERIODIC = 5   /* 1-D only: both ends of the line, joined */ };

/* Structured mesh of ni x nj cells (cell (i, j) -> index i + ni j). Vertex (i, j) is at index
 * i + (ni + 1) j of xv/yv ((ni+1)(nj+1) entries). dim = 1: a line of ni cells (nj = 1); only xv[0..ni]
 * is read and cells are unbounded in y. dim = 2: quadrilaterals (v(i,j), v(i+1,j), v(i+1,j+1), v(i,j+1))
 * counter-clockwise; periodic_j joins row nj to row 0 (O-mesh). Boundary tags: bc_imin/bc_imax have nj
 * entries, bc_jmin/bc_jmax ni entries (ignored when periodic_j or dim = 1). At most 2^21 - 1 cells. */
typedef struct {
    int32_t ni, nj, dim, periodic_j;
    const double* xv;
    const double* yv;
    const int32_t* bc_imin;
    const int32_t* bc_imax;
    const int32_t* bc_jmin;
    const int32_t* bc_jmax;
} ugkwp_mesh;

/* Unstructured mesh of triangles and convex quadrilaterals (the paper's meshes are unstructured, Sec. V).
 * cells: 4 vertex indices per cell, counter-clockwise, -1 in the fourth for a triangle. Local face k of a
 * cell is its edge from vertex k to vertex k + 1 (mod 3 or 4). Faces are numbered in order of first
 * appearance, walking the cells in order and each cell's edges in order; the first cell naming an edge is
 * the face's L side and the face keeps that cell's direction a -> b, so that its unit normal
 * (e_y, -e_x) / |e| points from L to R. boundary: 3 int32 per edge of a single cell (vertex, vertex in
 * either order, tag: wall, far field, fixed or symmetry), each such edge exactly once. Wall faces are
 * numbered in face order. Host arrays, read during ugkwp_create_unstructured only. */
typedef struct {
    int32_t n_vertices, n_cells;
    const double* xv;
    const double* yv;
    const int32_t* cells;
    int32_t n_boundary;
    const int32_t* boundary;
} ugkwp_umesh;

/* VHS exponent (mu ~ T^omega) and Prandtl number (Prandtl fix of the wave slopes; 1 = BGK) */
typedef struct {
    double omega, Pr;
    double wall_specular;     /* Maxwell wall: the fraction 1 - alpha of molecules (and of the incoming wave)
                                 reflected specularly, the rest re-emitted diffusely at T_w; 0 = fully diffuse
                                 (the default); in [0, 1] */
} ugkwp_gas;

typedef struct {
    uint64_t seed;            /* Philox key (low word xor case_id, high word) */
    uint32_t case_id;
    int32_t n_ref;            /* reference particles per cell, N_ref of Eq. 26 */
    int32_t precision;        /* 0: FP32 particles, FP32 interior wave fluxes and (first order) FP32 tau,
                                 e^{-dt/tau} of cells without a wall face; FP64 cell update, wall cells and
                                 wall fluxes; 1: everything FP64 */
    int32_t wave_only;        /* 1: no particles (GKS limit, deterministic) */
    int32_t record_faces;     /* 1: record, per face and step, the masses of the particles crossing it before
                                 and after the dt_R / dt_L scaling (the side-recorded fluxes of Sec. IV A,
                                 Eqs. 35-43), read by ugkwp_get_tallies; costs 32 F bytes and two 64-bit
                                 atomics per crossing. 0: off (the default). */
    int32_t capacity;         /* particle capacity; 0 = 4 n_ref cells */
    double ghost_state[4];    /* (rho, U, V, T) of UGKWP_BC_FIXED ghosts */
    void* stream;             /* cudaStream_t to run on (NULL: the legacy default stream) */
    int32_t use_graph;        /* 1: capture one step into a CUDA graph on the first ugkwp_step, replay it */
    int32_t order;            /* 2: second-order reconstruction of W and W^h for the wave fluxes (Eq. 12; 1-D a
                                 smooth van Albada-type limited slope, 2-D least squares with Venkatakrishnan's
                                 limiter; 128 B per cell); 0 or 1: first order (the default) */
    /* Device memory from the caller (both NULL: the library calls cudaMalloc / cudaFree itself). dev_alloc
     * returns `bytes` of device memory usable on `stream` (the context's stream), 256-byte aligned, or NULL
     * (the call then fails with ENOMEM); dev_free returns memory that dev_alloc gave. Every allocation of the
     * context goes through them: its state at creation, and the temporaries of the read-back and state-transfer
     * calls (returned before the call returns, after the context's stream has synchronised). The context frees
     * its state in ugkwp_destroy. Both must be set, or neither. */
    void* (*dev_alloc)(size_t bytes, void* stream, void* user);
    void (*dev_free)(void* ptr, void* user);
    void* alloc_user;         /* passed to dev_alloc and dev_free */
    double emx_cutoff;        /* particle cutoff (a reading of Sec. V A's cost discussion, which ties the cost of a
                                 step to the mass carried by particles): a cell whose collisionless fraction
                                 e^{-dt_i/tau_i} is below emx_cutoff samples no new particles that step, and its
                                 whole hydrodynamic part W^h then travels with the wave (free-transport weight
                                 dbar_d, as for a cell with rho^hp = 0). Such cells are wave-dominated: the ceil of
                                 Eq. 26 would give each of them one particle of negligible mass per step. Particles
                                 already in the cell (or arriving) are unaffected. 0: off (the default); in
                                 [0, 1), EINVAL otherwise. */
} ugkwp_opts;

/* Build the context: geometry, fixed local time steps (Eqs. 33-34), uniform freestream state, no
 * particles. Kn is the freestream mean free path over the mesh's length unit (VHS); Ma the freestream
 * Mach number along +x; Tw the wall temperature over T_inf; cfl the CFL number N_CFL of Eq. 33. */
ugkwp_status ugkwp_create(const ugkwp_mesh* mesh, const ugkwp_gas* gas, double Kn, double Ma, double Tw,
                          double cfl, ugkwp_tstep mode, const ugkwp_opts* opts, ugkwp_ctx** out);
/* As ugkwp_create on an unstructured mesh (at most 2^20 cells). UGKWP_EINVAL, with no context made, for a
 * vertex index out of range, a vertex repeated in a cell, a clockwise or non-convex cell, an edge of three
 * cells or of two cells running the same way along it, an untagged or twice-tagged boundary edge, a tag on
 * an interior edge, or a tag other than wall, far field, fixed and symmetry. Every other entry point works
 * on the context as on a structured one (cells in the given order, faces numbered as above). */
ugkwp_status ugkwp_create_unstructured(const ugkwp_umesh* mesh, const ugkwp_gas* gas, double Kn, double Ma,
                                       double Tw, double cfl, ugkwp_tstep mode, const ugkwp_opts* opts,
                                       ugkwp_ctx** out);
void ugkwp_destroy(ugkwp_ctx* ctx);

/* Advance n_steps steps (asynchronous). */
ugkwp_status ugkwp_step(ugkwp_ctx* ctx, int32_t n_steps);

/* out[4..7]: raw residual of the last step per conservative component (rho, rho U, rho V, rho E),
 * sqrt(sum_i Omega_i ((W^{n+1} - W^n) / dt_i)^2); out[0..3]: the same divided by a freestream scale that
 * cannot vanish, S_c sqrt(sum_i Omega_i) / L_ref with L_ref = 1, S = (rho c, rho c^2, rho c^2, rho c^3 / 2),
 * rho_inf = 1 and c = U_inf + sqrt(gamma R T_inf) (an O(1) imbalance of the freestream fluxes over the
 * whole domain reads about 1). The paper defines no residual (it judges steady state by monitored histories,
 * Sec. V A); this normalisation does not depend on what the first step changed, so a start whose first step
 * leaves a component unchanged (a plate's density) still has a meaningful 1e-6. Synchronises. */
ugkwp_status ugkwp_residual(ugkwp_ctx* ctx, double* out);

/* Wall pressure, shear stress (along t = (-n_y, n_x), n the outward normal of the fluid cell) and heat
 * flux into the wall on each of n_wall wall faces (in face order), either of the last step (averaged = 0)
 * or averaged over all steps since the last reset (averaged = 1). Synchronises. */
ugkwp_status ugkwp_surface(ugkwp_ctx* ctx, double* p, double* tau_w, double* q, int32_t n_wall,
                           int32_t averaged);
ugkwp_status ugkwp_reset_surface(ugkwp_ctx* ctx);
/* Monitored wall loads of the last step (Sec. V A: EMA histories of wall quantities judge the steady state;
 * Sec. V B: the drag coefficient), computed on the device at the end of every step: out[0] C_d = F_x /
 * (rho_inf U_inf^2 / 2) and out[1] C_H = Q / (rho_inf U_inf^3 / 2) with F = sum_j s_j (p_j n_j + tau_j t_j),
 * t = (-n_y, n_x), Q = sum_j s_j q_j over the wall faces (L_ref = 1); out[2] C_p = (p - p_inf) /
 * (rho_inf U_inf^2 / 2) and out[3] C_Q = q / (rho_inf U_inf^3 / 2) at the stagnation point, the mean of the
 * two wall faces whose normals face the freestream most (NaN when none faces it within 60 degrees, e.g. a
 * plate along the flow); out[4..7] their EMAs with alpha = 2/1001 from the first surface sample after
 * creation or ugkwp_reset_surface. NaN before the first step. Synchronises. out: 8 host doubles. */
ugkwp_status ugkwp_monitors(ugkwp_ctx* ctx, double* out);

/* Set the cell state from host primitives (rho, U, V, T) per cell (4 C doubles); removes all particles
 * (W^p = 0). The local time steps are unchanged. */
ugkwp_status ugkwp_set_field(ugkwp_ctx* ctx, const double* prim);
/* Replace the local time steps (C host doubles, each finite and > 0) from the next step on; the crossing
 * scaling dt_R / dt_L follows. A study tool for time-varying schedules (Sec. IV A, Eqs. 44-46): the method
 * itself keeps the steps of Eqs. 33-34 fixed, since stepwise scaling balances the time-averaged particle
 * fluxes only for fixed steps. Synchronises; EINVAL on a bad value (nothing changed). A captured step graph
 * stays valid (it reads the steps from device memory). */
ugkwp_status ugkwp_set_time_steps(ugkwp_ctx* ctx, const double* dt);
/* W (4 C doubles: rho, rho U, rho V, rho E) and, if Wp != NULL, W^p of the retained particles. */
ugkwp_status ugkwp_get_field(ugkwp_ctx* ctx, double* W, double* Wp);

/* ugkwp_get_field without allocating: the same values, with the W^p conversion in a fixed device scratch
 * array instead of a per-call temporary (the paper has no counterpart; it serves callers that must not
 * allocate, e.g. a monitor sampling a case while a batched launch runs on other streams, since cudaMalloc
 * and cudaFree synchronise the whole device). Limit for Wp != NULL: meshes of at most 98304 cells, else
 * EINVAL with a message (a W-only call, Wp == NULL, uses no scratch and serves any mesh). The context's
 * device must be the current device (else EINVAL). The scratch is shared by all calls on a device:
 * overlapping calls race, callers serialise them. The first call with Wp != NULL on a device looks the
 * scratch up; make it before any stream capture. Every check runs before a copy is queued, and a CUDA
 * error after that waits for the queued copies, so the host buffers are free again whenever it returns.
 * Synchronises. */
ugkwp_status ugkwp_get_field_noalloc(ugkwp_ctx* ctx, double* W, double* Wp);

/* out[13]: steps taken, particles, new in the last step, removed (collided), left the domain, face
 * crossings, wall hits, largest crossings + hits of one particle in the last step; then, cumulative since
 * creation, particle-steps processed (retained + new particles of every step) and new particles; then the
 * cells reset to the vacuum floor in the last step: a cell state outside the realizable set (density
 * above 1e-12, 0.01 min(1, T_w, T_fixed) <= T <= T_cap = 10 max(1 + Ma^2/3, T_w, T_fixed),
 * |U| <= U_inf + 10 sqrt(R T_cap)) restarts from rho = 1e-12 at rest at T_inf; a hydrodynamic part W^h
 * outside that set is not sampled and has no free-transport wave flux; last, the new particles of the
 * last step whose Shakhov acceptance-rejection (Pr != 1) kept a Maxwellian proposal after 64 rejections;
 * last, the particles that entered from far-field / fixed ghost sources in the last step. */
ugkwp_status ugkwp_stats(ugkwp_ctx* ctx, int64_t* out);
int64_t ugkwp_num_particles(ugkwp_ctx* ctx);

/* Particle snapshot to host arrays of length >= cap (values widened to double in FP32 mode). */
ugkwp_status ugkwp_get_particles(ugkwp_ctx* ctx, int64_t cap, uint64_t* pid, int32_t* cell, double* x,
                                 double* y, double* u, double* v, double* w, double* m);
/* Replace the whole state: step counter, W (4 C), the retained tally of the previous step (5 C int64,
 * fixed point, see ugkwp_fixed_exponents), and np particles (values must be FP32-representable in FP32
 * mode). */
ugkwp_status ugkwp_set_state(ugkwp_ctx* ctx, int64_t step, const double* W, const int64_t* wret, int64_t np,
                             const uint64_t* pid, const int32_t* cell, const double* x, const double* y,
                             const double* u, const double* v, const double* w, const double* m);
/* Integer tallies of the last step (any pointer may be NULL): W^{p,-} and W^{p,+} and the retained part
 * (5 C each: sum of m, m u, m v, m w, m |u|^2/2 in fixed point), face crossings (2 F: L->R, R->L),
 * wall momentum/energy transfer (3 per wall face), and the side-recorded crossing masses (4 F: per face,
 * L->R before and after the scaling, then R->L before and after; fixed point of the mass exponent; zeros
 * unless the context was created with record_faces = 1). */
ugkwp_status ugkwp_get_tallies(ugkwp_ctx* ctx, int64_t* wm, int64_t* wpl, int64_t* wret, int64_t* cross,
                               int64_t* wall, int64_t* frec);
/* Per cell (8 C doubles) of the last decomposition: tau, dt/tau, e^{-dt/tau}, N^hp, new-particle mass,
 * U^h, V^h, R T^h. */
ugkwp_status ugkwp_get_cell_data(ugkwp_ctx* ctx, double* out);
/* Time-averaged wave flux of the last step per face (4 F doubles, global frame, along the face normal). */
ugkwp_status ugkwp_get_flux(ugkwp_ctx* ctx, double* flux);
/* Local time steps and cell areas (C doubles each, nullable), face and wall-face counts (nullable). */
ugkwp_status ugkwp_get_geometry(ugkwp_ctx* ctx, double* dt, double* vol, int32_t* nfaces, int32_t* nwall);
/* Fixed-point exponents F of the mass, momentum and energy tallies: value = integer * 2^-F. */
ugkwp_status ugkwp_fixed_exponents(ugkwp_ctx* ctx, int32_t* out);
/* Batched launch: one CUDA graph that advances every listed context by one step per launch, each case's
 * kernels on streams of their own so that the cases' (latency-bound) kernels overlap on the GPU. The
 * contexts must be distinct, on the current device, and stay alive while the batch exists; their own
 * streams are ordered before and after each ugkwp_batch_step. `stream` (nullable) is the stream the graph
 * is launched on. Cases may differ in mesh, gas, Kn, Ma, T_w, mode and particle count. */
typedef struct ugkwp_batch ugkwp_batch;
ugkwp_status ugkwp_batch_create(ugkwp_ctx* const* ctxs, int32_t n, void* stream, ugkwp_batch** out);
/* Batched persistent kernel: one launch (captured in a CUDA graph) advances every listed context by one step.
 * The step's work is a device list of items (case, stage, blocks of that stage) in the step order of the
 * method (Sec. III C, Sec. IV B: decomposition, new particles, transport, sort, wave fluxes, update); the
 * launch's CTAs (ctas_per_sm x SMs; ctas_per_sm 4 or 6, 0 for 4) take items from a counter, and an item waits
 * (bounded, see ugkwp_batch_set_wait_limit) until its case's previous stage has finished, so that the stage
 * boundaries of one case overlap with other cases' work. Each item runs the same per-block arithmetic as the
 * step's own kernels: the results equal those of ugkwp_step on each context (particles as sets). Scope: every
 * context in production precision, first-order reconstruction, the warp-staged transport with 128-particle
 * tiles (ugkwp_set_launch transport 2, chunk 128), no per-stage profiling, all on one device, at most 64;
 * EINVAL otherwise (ugkwp_batch_create serves any context). The stage sizes that walk particles are planned from
 * each case's particle count at creation (any count gives the same results, only the balance changes).
 * Device memory (plan and control words) comes from the first context's allocator. */
ugkwp_status ugkwp_batch_create_persistent(ugkwp_ctx* const* ctxs, int32_t n, void* stream, int32_t ctas_per_sm,
                                           ugkwp_batch** out);
ugkwp_status ugkwp_batch_step(ugkwp_batch* batch, int32_t n_steps);
/* Persistent batches: the time limit of an item's wait for its case's previous stage (default 2 s); when it
 * runs out the CTA stops the batch: no CTA takes further items, every case's error word gets the limit bit
 * (their calls then report ELIMIT), the launch returns, and ugkwp_batch_status reports ELIMIT. The cases are
 * then in the middle of a step: restore them (ugkwp_load) before stepping again. `stall` != 0 is a test hook:
 * the step's last item then waits for one item more than its case's previous stage has, so that the limit is
 * sure to run out. Synchronises the batch's stream. */
ugkwp_status ugkwp_batch_set_wait_limit(ugkwp_batch* batch, int64_t limit_ns, int32_t stall);
/* Synchronises the batch's stream; ELIMIT (and in *where, nullable, case * 20 + stage of the wait that ran
 * out) once a persistent batch has stopped, else OK. */
ugkwp_status ugkwp_batch_status(ugkwp_batch* batch, int32_t* where);
/* out[4]: 1 for a persistent batch, its items per step, CTAs per launch, CTAs per SM (0 for a graph batch). */
ugkwp_status ugkwp_batch_plan(const ugkwp_batch* batch, int32_t* out);
void ugkwp_batch_destroy(ugkwp_batch* batch);

/* Checkpoint: the whole state (step counter, W, retained tally, particles, last residual,
 * particle-mass-ratio EMA, surface sums, monitors and counters) to a binary file, and back into a context created
 * with the same mesh, gas, mode, precision and options. Steps after ugkwp_load reproduce the uninterrupted
 * run (the particle draws are keyed by particle id and step). The local time steps are not part of the
 * state: a run that replaced them (ugkwp_set_time_steps) replaces them again after loading. Both
 * synchronise. */
ugkwp_status ugkwp_save(ugkwp_ctx* ctx, const char* path);
ugkwp_status ugkwp_load(ugkwp_ctx* ctx, const char* path);

/* Launch parameters of the particle kernels: the transport kernel (1: warp-chunked, every precision; 2:
 * warp-staged, production precision only, the default there: a stay pass in which each warp has the stay-test
 * fields of tiles of 128 particles (chunk 128; 64 otherwise) copied into its shared memory by bulk asynchronous
 * copies, double-buffered, and finishes the particles that only move, then a flight pass that flies the
 * queued rest, those with a face ahead or colliding, one per thread), the particles per chunk a warp claims (a
 * multiple of 32 in [32, 8192]; the warp-staged kernel's tile) and blocks per SM (1..16; the warp-staged stay
 * pass runs 4, 6 or 8), and the steps between counting sorts of the particles by
 * cell (1..64); 0 keeps a value. They change only the speed: both kernels perform the same per-particle
 * operations, chunks, tiles and sorts reorder particles, and every result is an integer sum or a
 * per-particle / per-face quantity. EINVAL for a value out of range or the warp-staged kernel in the FP64
 * mode. Takes effect at the next step (a captured step graph is re-captured); a batch keeps the values its
 * contexts had at ugkwp_batch_create. ugkwp_get_launch fills out[4]: chunk, blocks per SM, sort interval,
 * transport kernel. */
ugkwp_status ugkwp_set_launch(ugkwp_ctx* ctx, int32_t chunk, int32_t blocks_per_sm, int32_t sort_every,
                              int32_t transport);
ugkwp_status ugkwp_get_launch(ugkwp_ctx* ctx, int32_t* out);
/* Autotuner: times the warp-staged kernel (production precision; tiles of 64 particles at 6 or 8 blocks per SM,
 * of 128 at 4, 6 or 8) and the warp-chunked kernel with chunk {128, 256} x blocks per SM {4, 6, 8}, each with
 * sort interval {8, 16, 32}, over whole sort periods of at
 * least `steps` steps (real steps of the run: the state advances) with CUDA events on the context's stream,
 * keeps the fastest and returns it in best[4] (nullable, order of ugkwp_get_launch) and its milliseconds per
 * step in best_ms (nullable). Synchronises. A particle-free context keeps its values. */
ugkwp_status ugkwp_autotune(ugkwp_ctx* ctx, int32_t steps, int32_t* best, double* best_ms);

/* Per-stage device timing with CUDA events recorded on the context's stream around each stage of every
 * step taken while enabled (graph replay is bypassed meanwhile). ugkwp_profile synchronises, returns the
 * summed milliseconds of the 6 stages (ms[0..5]: decomposition + slot scan, new-particle sampling,
 * particle transport, tallies and compaction, ghost particle sources + wave fluxes, the periodic counting
 * sort of the particles by cell, conservative update + surface quantities + step bookkeeping) and the number
 * of profiled steps, and clears the record (ms needs room for 8 values). Profiled steps run the work of the
 * second stream (ghost sources and wave fluxes, otherwise overlapped with sampling and transport) on the
 * context's stream, so that each stage's time is its own; the results are the same. */
ugkwp_status ugkwp_set_profiling(ugkwp_ctx* ctx, int32_t enable);
ugkwp_status ugkwp_profile(ugkwp_ctx* ctx, double* ms, int64_t* steps);
/* ---- Learned warm start -------------------------------------------------------------------------------
 * A coordinate MLP maps a cell centroid and the case conditions (x, y, Kn, Ma, T_w) to an initial field
 * (log rho, u / U_inf, v / U_inf, log T). It only changes the field the steady LTS iteration (Sec. III C,
 * Sec. IV B) starts from: the local time steps stay those of the freestream (fixed at creation) and the
 * iteration is unchanged, so the converged state is the method's own. The paper has no such network; it is
 * an addition for fewer steps to steady state.
 *
 * Network: n_features inputs (>= 37), `depth` hidden SiLU layers of `width` units, n_out linear outputs.
 * Parameters are FP32 master values (one vector: every layer's weight matrix [out][in] row-major in layer
 * order, then every layer's bias in layer order); every product uses them rounded to BF16, with FP32
 * activations and accumulation. All device pointers below are caller-owned device memory; calls run on the
 * network's stream (ugkwp_mlp_create) unless stated otherwise. */
typedef struct ugkwp_mlp ugkwp_mlp;

/* Feature map of one geometry family: x^ = asinh((x - cx) / ell) / asinh(ext / ell), same for y with cy;
 * the features of a point are sin/cos(2^k pi x^), sin/cos(2^k pi y^) for k = 0..7 (32 values, in that
 * block order), x^, y^, log10 Kn, Ma and T_w each mapped linearly from [lo, hi] to [-1, 1], then zeros up
 * to n_features. */
typedef struct {
    double cx, cy, ell, ext;
    double kn_lo, kn_hi, ma_lo, ma_hi, tw_lo, tw_hi;
} ugkwp_feature_map;

/* params: host, ugkwp_mlp_num_params floats, or NULL for all zeros. EINVAL on bad sizes. */
ugkwp_status ugkwp_mlp_create(int32_t n_features, int32_t width, int32_t depth, int32_t n_out, const float* params,
                              void* stream, ugkwp_mlp** out);
void ugkwp_mlp_destroy(ugkwp_mlp* mlp);
int64_t ugkwp_mlp_num_params(const ugkwp_mlp* mlp);
/* Host copies of the parameters and of the gradient of the last ugkwp_mlp_grad (either may be NULL). */
ugkwp_status ugkwp_mlp_get_params(ugkwp_mlp* mlp, float* params, float* grad);
/* Replace the parameters from host memory; resets the Adam state. Synchronises. */
ugkwp_status ugkwp_mlp_set_params(ugkwp_mlp* mlp, const float* params);
/* y[n][n_out] = network(x[n][n_features]), device arrays. Asynchronous. */
ugkwp_status ugkwp_mlp_forward(ugkwp_mlp* mlp, const float* x, int32_t n, float* y);
/* Gradient of the mean squared error (1 / (n n_out)) sum (y - t)^2 over the points rows[0..n-1] of the
 * device arrays x[.][n_features] and t[.][n_out] (rows NULL: points 0..n-1), kept on the device for
 * ugkwp_mlp_adam; loss (host, nullable) receives the loss (then the call synchronises). Deterministic. */
ugkwp_status ugkwp_mlp_grad(ugkwp_mlp* mlp, const float* x, const float* t, const int32_t* rows, int32_t n,
                            float* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with learning rate lr on the last
 * gradient. Asynchronous. */
ugkwp_status ugkwp_mlp_adam(ugkwp_mlp* mlp, float lr);
/* Feature rows feat[n][n_features] of the points (x[i], y[i]) (device arrays; y NULL: 0) for one case's
 * conditions, on `stream`. */
ugkwp_status ugkwp_mlp_features(const ugkwp_feature_map* fmap, const double* x, const double* y, int32_t n,
                                double Kn, double Ma, double Tw, int32_t n_features, float* feat, void* stream);
/* acc[4 C] (device) = W (reset != 0) or acc + W: running sums of the conservative field for a time
 * average. On the context's stream. */
ugkwp_status ugkwp_field_accumulate(ugkwp_ctx* ctx, double* acc, int32_t reset);
/* Training pairs of every cell of a context: features of the cell centroids (feat[C][n_features]) and
 * targets (targ[C][4]) of the field W * scale, W a device array of 4 C conservative values (NULL: the
 * context's current field, scale ignored). On the context's stream. */
ugkwp_status ugkwp_mlp_dataset(ugkwp_ctx* ctx, const ugkwp_feature_map* fmap, const double* W, double scale,
                               int32_t n_features, float* feat, float* targ);
/* Set the context's field from the network at its cell centroids: rho = exp(y0) in [1e-6, 1e6],
 * (u, v) = U_inf (y1, y2) with speed at most U_cap / 2, T = exp(y3) in [2 T_min, T_cap / 2] (bounds as in
 * ugkwp_stats); removes all particles (W^p = 0), as ugkwp_set_field. Synchronises. n_out must be 4. */
ugkwp_status ugkwp_warm_start(ugkwp_ctx* ctx, ugkwp_mlp* mlp, const ugkwp_feature_map* fmap);

const char* ugkwp_last_error(const ugkwp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
