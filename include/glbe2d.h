/*
 * glbe2d.h -- C-ABI of the two-dimensional forms of the method in the GB300
 * (sm_103a) library: the preconditioned GLBE with forcing term on the D2Q9
 * lattice, optionally coupled to the preconditioned vector lattice kinetic
 * equation for the magnetic induction on the D2Q5 lattice (Premnath,
 * Pattison & Banerjee, arXiv:0809.4730, Secs. 2-4; the D2Q9 tables of App. A).
 *
 * One time step (glbe2d_step_n) is one fused kernel launch, one node (or, on
 * request, a pair of x-adjacent nodes; see variant) per thread:
 *   - rho = sum f, j = sum f e + F/(2 gamma) (Eq. precondhydrofields);
 *   - D2Q9 collision in moment space: the moment basis rho, e, e^2, j_x, q_x,
 *     j_y, q_y, p_xx, p_xy (App. A), equilibrium moments with every term
 *     quadratic in j divided by gamma (Sec. 3), the preconditioned source
 *     S* = P_S S with P_S = diag(1, g^-2, g^-2, g^-1, g^-1, g^-1, g^-1, g^-2,
 *     g^-2) (Eq. precondsourceterm), rates s_7 = s_8 = s_nu* with
 *     1/s_nu* = 3 nu/gamma + 1/2 and the kinetic rates of Sec. 3;
 *   - optional D2Q5 vector lattice (Sec. 4): N_m = 3, W_0 = 1/3, W_a = 1/6,
 *     theta_m = 1/3, tau_m* = eta/(gamma_m theta_m) + 1/2
 *     (Eq. mrelaxationtime), g^eq,* with the chi/gamma_m scaling of Sec. 4.1,
 *     B in the plane, J = J_z e_z with J_z = (1/(mu chi)) (d_x B_y - d_y B_x)
 *     from the non-equilibrium first moment, Lorentz force
 *     J x B = (-J_z B_y, J_z B_x) entering the next step's body force;
 *   - streaming (Eqs. pstreaming, mstreaming) with half-way bounce-back for f
 *     and anti-bounce-back to B0 (insulating walls) for g;
 *   - every 10th time level the residual r(t) = ||u(t) - u(t-10)|| / ||u(t)||
 *     over the fluid nodes with FP64 sums of mass and momentum (Sec. 5).
 *
 * Conventions (as in glbe.h, whose status codes, storage forms and residual
 * record this header reuses)
 *   - Lattice ordering (the paper lists the velocity groups only):
 *       D2Q9: 0 rest; 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1),
 *             7 (-1,-1), 8 (1,-1); weights 4/9, 1/9, 1/36.
 *       D2Q5: 0 rest; 1 +x, 2 -x, 3 +y, 4 -y.
 *   - Layout at this boundary: structure of arrays, [component][y][x] with x
 *     fastest, N = nx*ny.  g is [j][a][y][x] (component j of B, direction a).
 *     FP32 unless stated.
 *   - Populations crossing this boundary are deviations from the rest state,
 *     df_a = f_a - w_a rho0 and dg_ja = g_ja - W_a B0_j.
 *   - A node is solid when it lies on a wall line (wall_lo / wall_hi); its
 *     outputs are 0 and its inputs ignored.
 *   - The caller owns all device memory, including the workspace; the library
 *     never allocates device memory.  glbe2d_destroy frees host state only.
 *   - Every call enqueues on params.stream and returns without waiting, except
 *     glbe2d_residual, glbe2d_history, glbe2d_solve and glbe2d_sync.
 *   - Every call returns a glbe_status; glbe_last_error() holds the message.
 */
#ifndef GLBE2D_H
#define GLBE2D_H

#include <stddef.h>

#include "glbe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct glbe2d_ctx glbe2d_ctx;

typedef struct {
    int nx, ny;               /* grid, x fastest; N = nx*ny < 2^31                 */
    int wall_lo[2];           /* 1: the line at index 0 along x / y is solid (half-way wall at 0.5) */
    int wall_hi[2];           /* 1: the line at index n-1 is solid; 0 on both: periodic */
    double rho0;              /* reference density of the rest state               */
    double gamma;             /* flow preconditioning parameter, 0 < gamma <= 1     */
    double nu;                /* shear viscosity: rows 7, 8 relax at s_nu*, 1/s_nu* = 3 nu/gamma + 1/2 */
    double s[9];              /* rates of the other rows (default: s_1 = 1.63, s_2 = 1.14,
                                 s_4 = s_6 = 1.92 of Sec. 3; rows 0, 3, 5 are conserved and
                                 cannot change the result)                          */
    double F[2];              /* uniform body force                                 */
    int force_field;          /* 0: none; 2: a field [2][N] (glbe2d_set_force) added to F */
    int induction;            /* 1: couple the D2Q5 vector lattice                   */
    double gamma_m;           /* induction preconditioning parameter, 0 < gamma_m <= 1 */
    double eta;               /* magnetic diffusivity                               */
    double chi;               /* low-Pr_m scaling factor (Sec. 4.1), > 0            */
    double mu;                /* magnetic permeability, > 0                          */
    double B0[2];             /* applied in-plane field: initial state and wall value */
    int storage;              /* GLBE_F32, GLBE_BF16 or GLBE_F32C (glbe_storage)      */
    void* stream;             /* cudaStream_t owned by the caller                    */
    int variant;              /* kernel form: 0 = automatic (one node per thread, the plain step held
                                 to more resident blocks where that measured faster); 1 = one node
                                 per thread, free register allocation; 2 = two x-adjacent nodes per
                                 thread with vector loads and
                                 lane shuffles where x is periodic, nx even and the storage F32 or
                                 BF16 (else one node).  All forms give the same state bit for bit;
                                 the residual sums of form 2 agree to FP32 round-off */
} glbe2d_params;

/* Defaults: rho0 = 1, gamma = gamma_m = 1, chi = mu = 1, the D2Q9 kinetic
 * rates of Sec. 3 (conserved rows 1.0), eta = 0.1, F32 storage, no walls, no
 * force, no induction.  Grid and nu are left 0. */
void glbe2d_params_default(glbe2d_params* p);

/* Device workspace bytes glbe2d_init needs; GLBE_ERR_ARG for invalid
 * parameters (grid < 1 or N >= 2^31, a wall pair leaving no fluid line,
 * gamma, gamma_m outside (0, 1], nu, eta, chi, mu <= 0, a rate outside
 * (0, 2), a storage form other than F32, BF16, F32C, force_field not 0 or 2,
 * variant not 0, 1 or 2). */
glbe_status glbe2d_workspace_bytes(const glbe2d_params* p, size_t* bytes);

/* Creates a context on a caller-owned workspace (device memory of at least
 * glbe2d_workspace_bytes, 256-byte aligned) and enqueues the rest state
 * (df = dg = 0, Lorentz force 0, force field 0, t = 0).  *out is NULL on
 * failure. */
glbe_status glbe2d_init(const glbe2d_params* p, void* d_workspace, size_t bytes, glbe2d_ctx** out);

/* Copies a force field ([2][N] FP32, device) into the workspace
 * (force_field = 2 only, else GLBE_ERR_STATE). */
glbe_status glbe2d_set_force(glbe2d_ctx* ctx, const float* d_F);

/* Advances n >= 0 steps; the step colliding a level t with t % 10 == 0 also
 * evaluates the residual. */
glbe_status glbe2d_step_n(glbe2d_ctx* ctx, long n);

/* Synchronises and returns the latest residual record (momentum[2] = 0).
 * GLBE_ERR_DIVERGED if it saw a non-finite velocity. */
glbe_status glbe2d_residual(glbe2d_ctx* ctx, glbe_residual_info* out);

/* The most recent records, oldest first (at most the last 4096).  Syncs. */
glbe_status glbe2d_history(glbe2d_ctx* ctx, glbe_residual_info* out, long cap, long* n);

/* Marches until r(t) <= tol at a level t that is a multiple of 10, or until
 * max_steps steps were taken, replaying a CUDA graph of 10-step chunks whose
 * kernels stop on a device flag.  *steps_out = the converged level (or the
 * level reached), *r_out = its r.  GLBE_ERR_TIMEOUT / GLBE_ERR_DIVERGED as
 * glbe_solve.  Syncs. */
glbe_status glbe2d_solve(glbe2d_ctx* ctx, double tol, long max_steps, long* steps_out, double* r_out);

/* Fields of the current state as the next collision sees them: d_rho [N],
 * d_u [2][N] (u = j/rho with the half force, the Lorentz force included),
 * d_B [2][N] (induction only).  NULL outputs are skipped. */
glbe_status glbe2d_fields(glbe2d_ctx* ctx, float* d_rho, float* d_u, float* d_B);

/* Pre-collision state as deviations: d_df [9][N], d_dg [2][5][N] and d_FL
 * [2][N] (the lagged Lorentz force; induction only).  NULL outputs skipped. */
glbe_status glbe2d_get_state(glbe2d_ctx* ctx, float* d_df, float* d_dg, float* d_FL);

/* Replaces the state by these pre-collision deviations at level t >= 0
 * (NULL d_dg / d_FL keep those parts); clears the residual snapshot and
 * record and a divergence stop. */
glbe_status glbe2d_set_state(glbe2d_ctx* ctx, const float* d_df, const float* d_dg, const float* d_FL, long t);

/* Current time level. */
glbe_status glbe2d_time(const glbe2d_ctx* ctx, long* t);

/* Synchronises the context's stream; reports asynchronous CUDA errors. */
glbe_status glbe2d_sync(glbe2d_ctx* ctx);

/* Frees the host-side context (not the workspace).  NULL is ignored. */
void glbe2d_destroy(glbe2d_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif
