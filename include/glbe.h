/*
 * glbe.h -- C-ABI of the GB300 (sm_103a) library for the preconditioned
 * generalized lattice Boltzmann equation (GLBE) with forcing term, coupled to
 * the preconditioned D3Q7 vector lattice kinetic equation for the magnetic
 * induction (Premnath, Pattison & Banerjee, arXiv:0809.4730).
 *
 * One time step (glbe_step_n) is one fused kernel launch per node:
 *   - macroscopic fields rho = sum f, j = sum f e + F/(2 gamma)
 *     (Eq. precondhydrofields);
 *   - D3Q19 multiple-relaxation-time collision in moment space with the
 *     gamma-preconditioned equilibrium moments, the preconditioned source
 *     S* = P_S S and the rates Lambda* (Sec. 3, Eqs. ppostcollision,
 *     prelax_term, precondsourceterm; tables of App. A);
 *   - optional D3Q7 vector kinetic equation: B = sum g, g^eq,* with the chi
 *     scaling, J = (1/(mu chi)) curl B from the non-equilibrium first moment,
 *     Lorentz force J x B added to the body force (Sec. 4, Sec. 4.1);
 *   - streaming (Eqs. pstreaming, mstreaming) with half-way bounce-back walls
 *     for f and anti-bounce-back (insulating walls, B = B0) for g (Sec. 5);
 *   - every 10th time level: the velocity residual
 *     r(t) = ||u(t) - u(t-10)||_2 / ||u(t)||_2 with FP64 sums of mass and
 *     momentum (Sec. 5).
 *
 * Conventions
 *   - Lattice ordering (the paper lists the velocity groups only):
 *       D3Q19: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..10 = (1,1,0),(-1,1,0),
 *       (1,-1,0),(-1,-1,0); 11..14 = (1,0,1),(-1,0,1),(1,0,-1),(-1,0,-1);
 *       15..18 = (0,1,1),(0,-1,1),(0,1,-1),(0,-1,-1).
 *       D3Q7: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z.
 *   - Array layout at this boundary: structure of arrays, [component][z][y][x]
 *     with x fastest; N = nx*ny*nz.  g is [j][a][z][y][x] (component j of B,
 *     direction a).  All arrays passed in or out are FP32 unless stated.
 *   - Populations crossing this boundary are deviations from the rest state:
 *     df_a = f_a - w_a rho0 and dg_ja = g_ja - W_a B0_j.
 *   - A node is solid when it lies on a wall plane (wall_lo/wall_hi below);
 *     values of solid nodes in outputs are 0 and in inputs are ignored.
 *   - Memory: the caller owns every device buffer, including the workspace
 *     handed to glbe_init (size from glbe_workspace_bytes).  The library never
 *     allocates or frees device memory.  glbe_destroy frees host state only.
 *   - Streams: every call enqueues work on params.stream (a cudaStream_t,
 *     NULL = legacy default stream) and returns without waiting, except
 *     glbe_residual, glbe_solve and glbe_sync, which synchronise that stream.
 *   - Errors: every call returns a glbe_status; glbe_last_error() gives a
 *     thread-local message for the last failure.  No call aborts or throws.
 *   - A context is used from one host thread at a time; separate contexts are
 *     independent.
 */
#ifndef GLBE_H
#define GLBE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GLBE_ABI_VERSION 4

typedef struct glbe_ctx glbe_ctx;

typedef enum {
    GLBE_OK = 0,
    GLBE_ERR_ARG = 1,       /* invalid argument (sizes, pointers, parameters)       */
    GLBE_ERR_CUDA = 2,      /* a CUDA runtime call or kernel launch failed          */
    GLBE_ERR_DIVERGED = 3,  /* the residual became NaN/Inf (numerical instability)  */
    GLBE_ERR_TIMEOUT = 4,   /* glbe_solve hit max_steps before reaching tol         */
    GLBE_ERR_STATE = 5      /* call not valid in the context's current state        */
} glbe_status;

typedef enum {
    GLBE_F32 = 0,   /* deviations stored as FP32                                    */
    GLBE_BF16 = 1,  /* deviations stored as BF16 (round to nearest even), FP32 math */
    GLBE_F16 = 2,   /* deviations stored as FP16, times storage_scale, FP32 math    */
    GLBE_F32C = 3,  /* compensated: FP32 deviation plus an FP16 remainder (2^36
                       scaled), updated by an exact two-sum; FP32 math; 6 bytes
                       per population.  Corrections below one FP32 ulp of the
                       stored deviation accumulate instead of being dropped, which
                       removes the FP32 stagnation floor of steady solves.    */
    GLBE_BF16_SR = 4, /* BF16 deviations rounded stochastically (unbiased: rounded
                       away from zero with probability equal to the dropped
                       fraction of a unit in the last place), FP32 math; 2 bytes
                       per population.  Round-to-nearest drops every correction
                       below half a unit in the last place, so a steady march
                       freezes at a false fixed point (error ~ ulp / decay rate
                       of the slowest mode); stochastic rounding removes that
                       bias and leaves zero-mean noise of about one ulp.  The
                       random bits are counter-based (node, population, step),
                       so a march is reproducible.                            */
    GLBE_F16_SR = 5   /* FP16 deviations times storage_scale, rounded
                       stochastically as GLBE_BF16_SR                         */
} glbe_storage;

typedef struct {
    int nx, ny, nz;           /* grid; x fastest.  N = nx*ny*nz < 2^31          */
    int wall_lo[3];           /* 1: plane at index 0 along x/y/z is solid (half-way wall at 0.5) */
    int wall_hi[3];           /* 1: plane at index n-1 is solid; 0 on both: periodic */
    double rho0;              /* reference density of the rest state            */
    double gamma;             /* flow preconditioning parameter, 0 < gamma <= 1 (Sec. 3) */
    double nu;                /* shear viscosity: 1/s_nu* = 3 nu/gamma + 1/2 on rows 9,11,13,14,15 (Sec. 3) */
    double s[19];             /* relaxation rates of the other rows (kinetic rates of Sec. 3 by default;
                                 rows 0,3,5,7 are conserved and cannot change the result) */
    double F[3];              /* uniform external body force                     */
    int force_field;          /* 0: none; 1: F_x field [N]; 3: field [3][N]; added to F */
    int induction;            /* 1: couple the D3Q7 vector lattice (Sec. 4)       */
    double gamma_m;           /* induction preconditioning parameter, 0 < gamma_m <= 1 */
    double eta;               /* magnetic diffusivity: tau_m* = eta/(gamma_m theta_m) + 1/2 (Eq. mrelaxationtime) */
    double chi;               /* low-Pr_m scaling factor chi > 0 (Sec. 4.1)      */
    double mu;                /* magnetic permeability                           */
    double B0[3];             /* applied field: initial state and wall value      */
    int storage;              /* glbe_storage                                    */
    double storage_scale;     /* F16 and F16_SR: multiplier on the stored deviations (0 = default 4096);
                                 ignored for the other storage forms */
    void* stream;             /* cudaStream_t owned by the caller                */
    int variant;              /* kernel form: 0 = automatic (on grids without walls along x and an even
                                 nx, without induction, with BF16 or F16 storage: the paired form,
                                 as measured faster; else one node per thread; with induction the F32C
                                 steps and the F32 and BF16 residual steps update a node in two
                                 passes, induction then flow, on grids of more than two resident
                                 waves, and so do the FP32 cavity steps: the one-pass results bit for
                                 bit);
                                 1 = one node per thread; 2 = two x-adjacent
                                 nodes per thread with packed FP32x2 arithmetic (needs an even nx and
                                 no walls along x, else the one-node form is used); 3 = tiles of 128
                                 x-nodes whose gathers are staged in shared memory by tensor-memory
                                 copies (needs no walls along x, nx a multiple of 128, F32, BF16 or
                                 F16 storage, not the _SR forms; else the one-node form is used); 4 = the same tiles with
                                 two x-adjacent nodes per thread in packed FP32x2 arithmetic */
    int collision;            /* 0 (default): the MRT-GLBE (Secs. 2-3).  1: its limiting form, the preconditioned
                                 SRT-LBE with forcing term (Sec. 3.1): all rates 1/tau* = s_nu*, equilibrium
                                 f^eq,* and source S* of Eq. precondsourcecorrect in particle velocity space.
                                 2: the same SRT with the naive source of Eq. precondsourceincorrect, whose
                                 Chapman-Enskog expansion has a spurious momentum term for gamma < 1 (for
                                 comparison).  1 and 2 take F32, F32C or BF16 storage and run one node per
                                 thread; the batch and the adjoint take 0 */
    int box;                  /* 1: the flow lattice is fluid only on nodes with box_lo <= c <= box_hi (per axis,
                                 inclusive; outside, up to the wall planes, the induction lattice
                                 continues at rest: an extended magnetic domain whose wall planes
                                 hold the induced field at zero, Sec. 5, MHD cavity).  0: the whole
                                 grid off the wall planes is fluid */
    int box_lo[3], box_hi[3];
    double U_lid[3];          /* velocity of the flow boundary above the highest fluid z plane (the
                                 moving lid of the cavity, Sec. 5): a link bounced there returns
                                 with 6 w_a rho0 (e_a . U_lid) added (Ladd's moving-wall rule).
                                 A box or a non-zero lid runs the one-node cavity kernel (F32,
                                 F32C or BF16 storage; the MRT or, with F32, the SRT collision);
                                 glbe_get_state / glbe_set_state, the batch and the adjoint do not
                                 take it */
    int ghost_lo, ghost_hi;   /* slab decomposition along z.  1: the plane z = 0 (resp. z = nz-1) is a ghost
                                 plane holding what the neighbouring slab streams across the face
                                 (glbe_halo_unpack): it is never collided, is outside every sum and
                                 output (like a solid plane), and a gather reads it as fluid.  Not
                                 together with a wall on the same side.  0 (default): no ghost plane */
} glbe_params;

/* Latest residual evaluation (time level t, a multiple of 10). */
typedef struct {
    long t;                   /* time level of u(t); -1 if none evaluated yet    */
    double r;                 /* ||u(t)-u(t-10)|| / ||u(t)|| over fluid nodes   */
    double num, den;          /* sum |u(t)-u(t-10)|^2 and sum |u(t)|^2 (FP64)    */
    double mass;              /* sum rho over fluid nodes (FP64)                 */
    double momentum[3];       /* sum rho u over fluid nodes (FP64)               */
    int nonfinite;            /* number of fluid nodes with a NaN/Inf velocity   */
} glbe_residual_info;

/* Fills p with the defaults: rho0 = 1, gamma = gamma_m = 1, chi = mu = 1,
 * the kinetic rates of Sec. 3 (s1 = 1.19; s2 = s10 = s12 = 1.4;
 * s4 = s6 = s8 = 1.2; s16..18 = 1.98; conserved rows 1.0), F32 storage,
 * no walls, no force, no induction.  Grid and nu are left 0. */
void glbe_params_default(glbe_params* p);

/* Bytes of device workspace glbe_init needs for these parameters.
 * Returns GLBE_ERR_ARG for invalid parameters. */
glbe_status glbe_workspace_bytes(const glbe_params* p, size_t* bytes);

/* Creates a context on the caller's workspace (device memory of at least
 * glbe_workspace_bytes, 256-byte aligned) and enqueues the rest-state
 * initialisation (df = 0, dg = 0, Lorentz force 0, t = 0).  The workspace
 * must stay allocated until glbe_destroy.  *out is NULL on failure. */
glbe_status glbe_init(const glbe_params* p, void* d_workspace, size_t bytes, glbe_ctx** out);

/* Copies the body-force field (device, FP32, force_field components, layout
 * [comp][z][y][x]) into the workspace.  The field is added to params.F.
 * The source may be freed after the copy completes on the stream. */
glbe_status glbe_set_force(glbe_ctx* ctx, const float* d_F);

/* Same from host memory.  The field applies to the steps enqueued after this
 * call.  The host copy goes to a staging region of the workspace on the
 * library's own copy stream, so it overlaps the steps already enqueued on the
 * context's stream; that stream then waits for it and moves the field in with
 * a device copy.  Pinned memory makes the host copy asynchronous.  The host
 * buffer must stay valid until the copy completes, which is at the latest
 * when the context's stream reaches the steps enqueued after this call. */
glbe_status glbe_set_force_host(glbe_ctx* ctx, const float* h_F);

/* Advances n >= 0 time steps (one fused kernel per step; the residual is
 * evaluated inside the step that collides a level t with t % 10 == 0). */
glbe_status glbe_step_n(glbe_ctx* ctx, long n);

/* Synchronises the stream and returns the latest residual evaluation.
 * GLBE_ERR_DIVERGED if it saw a non-finite velocity. */
glbe_status glbe_residual(glbe_ctx* ctx, glbe_residual_info* out);

/* Copies the most recent residual evaluations (oldest first) into out[0..cap),
 * at most the last 4096 kept on the device; *n = number copied.
 * Synchronises the stream. */
glbe_status glbe_history(glbe_ctx* ctx, glbe_residual_info* out, long cap, long* n);

/* Time-marches until r(t) <= tol (t a multiple of 10) or max_steps steps have
 * been taken, replaying a CUDA graph of 10-step chunks.  *steps_out = time
 * level t of the converged residual (or the level reached), *r_out = r(t).
 * GLBE_ERR_TIMEOUT if max_steps was reached first, GLBE_ERR_DIVERGED on
 * NaN/Inf.  Synchronises the stream. */
glbe_status glbe_solve(glbe_ctx* ctx, double tol, long max_steps, long* steps_out, double* r_out);

/* Macroscopic fields of the current state, as the next collision sees them
 * (rho, u = j/rho with the half-force, B = sum g).  d_rho [N], d_u [3][N],
 * d_B [3][N] (ignored and may be NULL without induction).  Any output may be
 * NULL. */
glbe_status glbe_fields(glbe_ctx* ctx, float* d_rho, float* d_u, float* d_B);

/* Current pre-collision state as deviations: d_df [19][N], d_dg [3][7][N]
 * (induction only), d_FL [3][N] Lorentz force of the last step (induction
 * only).  NULL outputs are skipped. */
glbe_status glbe_get_state(glbe_ctx* ctx, float* d_df, float* d_dg, float* d_FL);

/* Replaces the state by the given pre-collision deviations (layout as in
 * glbe_get_state; NULL d_dg / d_FL leave those parts unchanged) at time
 * level t >= 0.  Clears the residual snapshot, the residual record and a
 * divergence stop left by an earlier non-finite residual. */
glbe_status glbe_set_state(glbe_ctx* ctx, const float* d_df, const float* d_dg, const float* d_FL, long t);

/* Checkpoint / resume (the paper has no counterpart; a service of the
 * library).  A checkpoint is one host buffer holding the raw state of the
 * context: the populations in the storage type, the lagged Lorentz force,
 * the force field, the velocity snapshot of the residual, the residual record,
 * the time level and the residual counters.  Loading it into a context with
 * the same grid, storage, coupling and force_field makes the following march
 * bit for bit the one the saved context would have made (the residual history
 * restarts empty).  Both calls synchronise the stream; the buffer is plain
 * (pageable or pinned) host memory owned by the caller.  glbe_checkpoint_load
 * returns GLBE_ERR_ARG for a buffer of another shape or library version. */
glbe_status glbe_checkpoint_bytes(const glbe_ctx* ctx, size_t* bytes);
glbe_status glbe_checkpoint_save(glbe_ctx* ctx, void* h_buf, size_t bytes);
glbe_status glbe_checkpoint_load(glbe_ctx* ctx, const void* h_buf, size_t bytes);

/* Current time level. */
glbe_status glbe_time(const glbe_ctx* ctx, long* t);

/* Synchronises the context's stream; reports asynchronous CUDA errors. */
glbe_status glbe_sync(glbe_ctx* ctx);

/* Message of the last failed call on this host thread ("" if none). */
const char* glbe_last_error(void);

/* Frees the host-side context (not the workspace). NULL is ignored. */
void glbe_destroy(glbe_ctx* ctx);

/* Allocation-free time step (the paper has no counterpart; this is a service
 * of the library).  For callers that cannot call cudaMalloc -- e.g. code whose
 * device memory is owned by another allocator (a framework's pool or a fixed
 * arena) and that may not allocate itself -- and so cannot provide the
 * workspace of glbe_init.  It performs one fused D3Q19 time step with the
 * residual evaluation on buffers the caller already holds:
 *   p          parameters as for glbe_init (induction must be 0; p->stream is
 *              used and synchronised)
 *   d_src      populations entering the step, d_dst populations leaving it:
 *              the library's own buffer layout, i.e. the deviations in the
 *              storage type, [19][N] (F32C: 19N FP32 high parts followed by
 *              19N FP16 low parts); all-zero bytes are the rest state.  The
 *              next step takes d_dst as its d_src.
 *   d_force    the force field ([force_field][N] FP32) or NULL if force_field = 0
 *   d_u        [3][N] FP32: on entry u of the previous evaluation (read only if
 *              have_prev), on exit u of the level t being collided
 *   t          time level being collided (only recorded in *out)
 *   out        host: the residual sums against d_u's entry values
 *              (out->t = -1 when have_prev = 0)
 * Its scratch (per-block partial sums and one record, about 1 MiB) is a
 * file-scope static array in the library's device memory, held by every GPU
 * that loads the library until the process exits.  The first call on a device
 * looks up that array's device address; make this first call before any
 * stream capture.  The address is kept per device and per driver context: after
 * cudaDeviceReset (or when the device's primary context is released and
 * created again) the next call looks it up anew, so make that call, too,
 * outside any stream capture.  Every call shares the array, so calls that
 * overlap on the GPU (other threads or streams) race and must be serialised by
 * the caller.  With variant 3 or 4, GLBE_ERR_TIMEOUT reports that a bounded
 * pipeline wait of the TMA-staged kernel ran out (the outputs are then
 * incomplete).  The residual record is read back on p->stream.
 * Grids of more than 4,194,304 nodes (16384 blocks of 256) and buffers that
 * are not 16-byte aligned are rejected with GLBE_ERR_ARG.  No call to cudaMalloc, cudaFree or any allocating routine is
 * made. */
glbe_status glbe_step_residual_noalloc(const glbe_params* p, const void* d_src, void* d_dst, const float* d_force,
                                       float* d_u, int have_prev, long t, glbe_residual_info* out);

/* ------------------------------------------------------------------------ */
/* Batched steady solves: many independent lattices (own grid, walls, gamma, */
/* rates, with or without the induction lattice) marched together by one    */
/* persistent cooperative kernel (one node per thread over a flattened tile  */
/* list, a bounded grid barrier between steps), launched from a CUDA graph.  */
/* Every 10 levels each domain's residual is reduced in a fixed order; a     */
/* domain whose r(t) <= tol leaves the march with its level and the device   */
/* time since the start of the launch.  Storage F32 or F32C, uniform force.  */
/* ------------------------------------------------------------------------ */
#define GLBE_BATCH_MAX_DOMAINS 4096

typedef struct glbe_batch glbe_batch;

typedef struct {
    int converged;            /* 1: r(t) <= tol was reached                      */
    long steps;               /* level t of that residual (-1 if not converged) */
    double r;                 /* last residual of the domain                     */
    double seconds;           /* device time from the start of the launch to the
                                 domain's convergence (-1 if not converged)      */
    int nonfinite;            /* 1: the domain's velocity became NaN/Inf         */
} glbe_batch_result;

/* Workspace bytes for n domains (each glbe_params as for glbe_init; the
 * stream field is ignored, force_field must be 0, all domains share one
 * storage type, F32 or F32C). */
glbe_status glbe_batch_workspace_bytes(const glbe_params* domains, int n, size_t* bytes);

/* Creates a batch on a caller-owned, 256-byte aligned workspace and sets every
 * domain to the rest state.  stream: cudaStream_t for all batch work.
 * Synchronises the stream. */
glbe_status glbe_batch_init(const glbe_params* domains, int n, void* d_workspace, size_t bytes, void* stream,
                            glbe_batch** out);

/* Launch shape of the persistent kernel: block_threads 128 or 256 (also the
 * tile size), blocks_per_sm from 1 to the occupancy limit. */
glbe_status glbe_batch_set_launch(glbe_batch* b, int block_threads, int blocks_per_sm);

/* Times steps_per_trial steps for every (block_threads, blocks_per_sm)
 * candidate on the batch itself, keeps the fastest and restores the rest
 * state.  Outputs may be NULL. */
glbe_status glbe_batch_autotune(glbe_batch* b, int steps_per_trial, int* block_threads, int* blocks_per_sm,
                                double* seconds_per_step);

/* Marches all domains from the rest state until each has r(t) <= tol or
 * max_steps levels have been taken, in one persistent launch (captured in a
 * CUDA graph when use_graph != 0).  results[n]; *seconds = device time of the
 * whole launch (may be NULL).  GLBE_ERR_TIMEOUT if some domain did not
 * converge or the grid barrier timed out, GLBE_ERR_DIVERGED on NaN/Inf,
 * GLBE_ERR_STATE if the batch was already solved (see glbe_batch_reset).
 * Synchronises the stream. */
glbe_status glbe_batch_solve(glbe_batch* b, double tol, long max_steps, int use_graph, glbe_batch_result* results,
                             double* seconds);

/* Macroscopic fields of domain d after a solve (layout as glbe_fields). */
glbe_status glbe_batch_fields(glbe_batch* b, int d, float* d_rho, float* d_u, float* d_B);

/* Returns every domain to the rest state for a new solve. */
glbe_status glbe_batch_reset(glbe_batch* b);

/* Failure detection: every wait of the batch's grid barrier gives up after
 * spin_limit polls (default 2^26, about 4 s), sets an error flag and ends the
 * launch (glbe_batch_solve then returns GLBE_ERR_TIMEOUT).  absent_block >= 0
 * makes that block leave the launch at once so that tests can drive the wait
 * to its limit without faulting or hanging the GPU; -1 (default) disables it. */
glbe_status glbe_batch_set_barrier_test(glbe_batch* b, long long spin_limit, int absent_block);

/* Frees the host-side batch (not the workspace). NULL is ignored. */
void glbe_batch_destroy(glbe_batch* b);

/* ------------------------------------------------------------------------ */
/* Gradient of a velocity objective with respect to the body force (the     */
/* paper has no adjoint; this differentiates its time step).                 */
/*   Q = sum over fluid nodes x of w(x) . u(x), u = j/rho with the half     */
/*   force (Eq. precondhydrofields).  d_w is [3][N] FP32 or NULL for the    */
/*   flow rate Q = (1/L_x) sum_fluid u_x (L_x = fluid planes along x).      */
/*   d_dQdF receives dQ/dF(x), [3][N] FP32, for a force field of three       */
/*   components added to params.F (0 on solid nodes), whatever the          */
/*   context's force_field.                                                  */
/* The state that is differentiated is the pre-collision f, g and the lagged */
/* Lorentz force, as in glbe_get_state; one adjoint step applies the         */
/* transposed node update (collision, Lorentz coupling, Secs. 2-4) after the */
/* transposed streaming (bounce-back / anti-bounce-back walls), one thread   */
/* per node.  Storage must be GLBE_F32 or GLBE_F32C (GLBE_ERR_ARG else).     */
/* The caller provides the workspace (glbe_adjoint_workspace_bytes,         */
/* 256-byte aligned device memory); nothing is allocated.  All work runs on  */
/* the context's stream.                                                     */
/* ------------------------------------------------------------------------ */

/* Workspace bytes of glbe_adjoint_steady (nsteps = 0) or of
 * glbe_adjoint_unrolled(nsteps, K): two cotangent buffers of 43N floats plus,
 * for the steady form, the linearisation rows of the fixed state (16N floats
 * with induction, 7N without: the forward quantities the transposed update
 * needs, written once per call), and for the unrolled form ceil(nsteps/K)
 * checkpoints and min(K, nsteps) recomputed states (each a population buffer
 * pair and the Lorentz force). */
glbe_status glbe_adjoint_workspace_bytes(const glbe_params* p, long nsteps, long K, size_t* bytes);

/* Steady adjoint at the context's current state, which should be a converged
 * steady state (glbe_solve): iterates lam <- J^t lam + dQ/ds, J the Jacobian
 * of one time step there, until the gradient field changes by at most tol
 * over 10 iterations, r = ||dQdF_k - dQdF_{k-10}|| / ||dQdF_k||, or max_iters
 * (>= 10) is reached.  Mass is conserved by the step, so lam may drift along
 * the uniform mode of f; that mode does not enter dQ/dF (the force adds no
 * mass).  *iters_out = iterations at the last evaluation, *r_out = its r.
 * GLBE_ERR_TIMEOUT if max_iters came first (d_dQdF then holds the last
 * iterate), GLBE_ERR_DIVERGED on NaN/Inf.  The state is not changed.
 * Synchronises the stream. */
glbe_status glbe_adjoint_steady(glbe_ctx* ctx, const float* d_w, double tol, long max_iters, void* d_work,
                                size_t bytes, float* d_dQdF, long* iters_out, double* r_out);

/* Unrolled adjoint: marches the context nsteps >= 1 steps from its current
 * level t0 (as glbe_step_n; the context ends at t0 + nsteps), keeping a
 * checkpoint every K >= 1 levels, then sweeps backwards segment by segment
 * (each segment recomputed from its checkpoint) and writes dQ/dF of Q taken
 * on the final state.  Enqueued asynchronously on the stream. */
glbe_status glbe_adjoint_unrolled(glbe_ctx* ctx, const float* d_w, long nsteps, long K, void* d_work, size_t bytes,
                                  float* d_dQdF);

/* ------------------------------------------------------------------------ */
/* Slab decomposition along z (the update is local except nearest-neighbour  */
/* streaming, Eqs. pstreaming and mstreaming): a grid is split into slabs of */
/* z planes, each a context with ghost planes (glbe_params.ghost_lo/hi).     */
/* After every step, the populations that cross a face -- the 5 D3Q19       */
/* directions with e_z = +-1 and, with induction, the D3Q7 direction e_z =   */
/* +-1 of each of the 3 components -- go from the slab's outermost computed  */
/* plane into the neighbour's ghost plane: glbe_halo_pack on one side, a     */
/* copy of the packed buffer (same device, a peer device or another process  */
/* by a collective library), glbe_halo_unpack on the other.  The lagged      */
/* Lorentz force is local.  A march of slabs is then bit for bit the march  */
/* of the whole grid.                                                        */
/* ------------------------------------------------------------------------ */

/* Bytes of one packed face: (5 + 3 with induction) rows of nx*ny values in
 * the storage type; the compensated form appends the FP16 low parts of the
 * same rows.  Layout: f rows, g rows, then (F32C) f low rows, g low rows;
 * rows in direction order. */
glbe_status glbe_halo_bytes(const glbe_ctx* ctx, size_t* bytes);

/* Packs (device buffer d_buf of glbe_halo_bytes) the post-collision
 * populations of the current level that leave through face 1 (high z: the
 * e_z = +1 directions of plane nz-2) or face 0 (low z: the e_z = -1
 * directions of plane 1).  The face must have a ghost plane.  Enqueued on the
 * context's stream. */
glbe_status glbe_halo_pack(glbe_ctx* ctx, int face, void* d_buf);

/* Writes a neighbour's packed face into this slab's ghost plane: face 0 (z =
 * 0) takes the neighbour's face-1 pack (e_z = +1 directions), face 1 (z =
 * nz-1) its face-0 pack.  Enqueued on the context's stream; the buffer must
 * hold the data when the stream reaches the copy. */
glbe_status glbe_halo_unpack(glbe_ctx* ctx, int face, const void* d_buf);

/* Combines the residual records of the n slabs of one grid taken at the same
 * level (sums of num, den, mass, momentum and non-finite counts, added in
 * FP64 in slab order) into the record of the grid, r = sqrt(num / den).
 * GLBE_ERR_ARG if the levels differ. */
glbe_status glbe_residual_combine(const glbe_residual_info* parts, int n, glbe_residual_info* out);

/* ABI version of the loaded library (GLBE_ABI_VERSION). */
int glbe_abi_version(void);

/* sizeof(glbe_params) and sizeof(glbe_residual_info) as compiled into the
 * library, so that bindings can verify their struct mirrors. */
void glbe_struct_sizes(size_t* params_bytes, size_t* info_bytes);

#ifdef __cplusplus
}
#endif

#endif /* GLBE_H */
