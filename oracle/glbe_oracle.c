/*
 * glbe_oracle.c -- plain FP64 CPU oracle of the preconditioned generalized
 * lattice Boltzmann equation (GLBE) with forcing term (D3Q19, multiple
 * relaxation times), coupled to the preconditioned D3Q7 vector lattice kinetic
 * equation for the magnetic induction (Premnath, Pattison & Banerjee,
 * "Steady state convergence acceleration of the generalized lattice Boltzmann
 * equation with forcing term through preconditioning", arXiv:0809.4730).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  The CUDA library never
 * calls it and shares no code, header, table or constant with it.
 *
 * Design rules of this file:
 *   - IEEE FP64 throughout, fixed loop order, no fast-math and no FMA
 *     contraction (the build passes -ffp-contract=off) so that x86 and Arm
 *     hosts produce identical bits.
 *   - The moment matrix T is built from its defining polynomials and applied as
 *     a dense 19x19 product; its inverse is T^t D^-1 (orthogonal rows).  No
 *     common-subexpression form, no fusion: every step follows the paper's
 *     order and notation so it can be checked by eye.
 *   - Storage is array-of-structures: f[n*19+a], g[n*21+j*7+a], FL[n*3+i],
 *     with node n = (z*ny + y)*nx + x.
 *   - Streaming is a push: the post-collision value of node n travels to
 *     n + e_a; a link that ends in a solid node is bounced back (half-way).
 *
 * Readings of the paper used here (where it is silent or inconsistent):
 *   - D3Q19 ordering (the paper gives groups only, Eq. velocityd3q19):
 *       0 rest; 1..6 = +x,-x,+y,-y,+z,-z;
 *       7..10 = (1,1,0),(-1,1,0),(1,-1,0),(-1,-1,0);
 *       11..14 = (1,0,1),(-1,0,1),(1,0,-1),(-1,0,-1);
 *       15..18 = (0,1,1),(0,-1,1),(0,1,-1),(0,-1,-1).
 *     Weights 1/3, 1/18, 1/36 (the standard D3Q19 set the paper cites).
 *   - D3Q7 ordering 0 rest, 1..6 = +x,-x,+y,-y,+z,-z; W_0 = 1/4, W_a = 1/8,
 *     theta_m = 1/4 (Sec. 4, N_m = 4).
 *   - The collision of the vector equation (Eq. mcollision) is printed without
 *     the "g +" term; the relaxation g~ = g - (g - g^eq)/tau_m is used.
 *   - Current density: the printed index order of Eq. for J gives -(1/mu)curl B
 *     once App. C's Lambda^(1)_ji = -tau theta d_j B_i is inserted, contrary to
 *     the definition J = (1/(mu chi)) curl B beside it.  The definition is
 *     kept: J_i = -(1/(mu chi tau_m theta_m)) eps_ijk Lneq_jk with
 *     Lneq_jk = sum_a e_aj (g_ak - g^eq_ak).
 *   - Coupling order within a time step: the Lorentz force of the previous
 *     step (stored per node) enters the half-force shift of the velocity used
 *     in g^eq; the new Lorentz force J x B is then formed and used for the
 *     fluid's half-force, equilibrium and source.  At a steady state both
 *     forces coincide, so the fixed point is the implicit one.
 *   - Insulating walls for the induction lattice: anti-bounce-back
 *     g_abar(x_f, t+1) = -g~_a(x_f, t) + 2 W_a B_wall (B_wall = applied field).
 *   - Residual: r(t) = ||u(t) - u(t-10)||_2 / ||u(t)||_2 over fluid nodes and
 *     all three components, evaluated when the state of time level t (a
 *     multiple of 10) is collided.
 *   - Moving wall (Sec. 5, 3D cavity: link bounce-back with the wall's
 *     momentum, Ladd): a post-collision population f~_a of a fluid node whose
 *     link ends on the moving lid returns as f_abar = f~_a - 2 w_a rho0
 *     (e_a . U)/c_s^2 = f~_a - 6 w_a rho0 (e_a . U).  The preconditioned
 *     equilibrium keeps the unscaled linear term 3 e.j, so the wall term is
 *     the one of the plain scheme.  The lid is the flow boundary above the
 *     highest fluid z plane.
 *   - Extended induction domain (Sec. 5, MHD cavity: the induced field is
 *     zero far from the cavity): the flow lattice is fluid only inside a box
 *     of nodes; around it, up to the wall planes of the grid, the vector
 *     lattice continues with u = 0 and no Lorentz force (pure magnetic
 *     diffusion), and the zero induced field is imposed at the grid's wall
 *     planes by the same anti-bounce-back to B0 as the insulating walls.
 */
#include <math.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------- */
/* Parameters (the oracle's own struct; mirrors what the paper specifies)  */
/* ---------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    int wall_lo[3], wall_hi[3];  /* 1: the plane at index 0 / n-1 is solid  */
    double rho0;                 /* reference density (initial state)       */
    double gamma;                /* flow preconditioning parameter, Sec. 3   */
    double nu;                   /* shear viscosity -> s_nu*, Sec. 3         */
    double s[19];                /* rates of the non-viscous rows; rows 9,11,13,14,15 are overwritten by s_nu* */
    double F[3];                 /* uniform external force, added to the field */
    int induction;               /* 1: couple the D3Q7 vector lattice        */
    double gamma_m;              /* induction preconditioning parameter      */
    double eta;                  /* magnetic diffusivity -> tau_m*, Eq. mrelaxationtime */
    double chi;                  /* low-Pr_m scaling factor, Sec. 4.1        */
    double mu;                   /* magnetic permeability                    */
    double B0[3];                /* applied field: initial state and wall value */
    int box;                     /* 1: the flow lattice is fluid only for box_lo <= c <= box_hi */
    int box_lo[3], box_hi[3];    /* (inclusive, per axis); the vector lattice covers every node off the walls */
    double U_lid[3];             /* velocity of the flow boundary above the highest fluid z plane */
} orc_params;

int orc_params_size(void) { return (int)sizeof(orc_params); }

/* ---------------------------------------------------------------------- */
/* Lattices                                                                */
/* ---------------------------------------------------------------------- */
static const int E19[19][3] = {
    {0,0,0},
    {1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1},
    {1,1,0},{-1,1,0},{1,-1,0},{-1,-1,0},
    {1,0,1},{-1,0,1},{1,0,-1},{-1,0,-1},
    {0,1,1},{0,-1,1},{0,1,-1},{0,-1,-1}};

static const int E7[7][3] = {
    {0,0,0},{1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1}};

static double w19(int a)
{
    int c2 = E19[a][0]*E19[a][0] + E19[a][1]*E19[a][1] + E19[a][2]*E19[a][2];
    return c2 == 0 ? 1.0/3.0 : (c2 == 1 ? 1.0/18.0 : 1.0/36.0);
}

static const double THETA_M = 0.25;          /* theta_m = 1/N_m, N_m = 4 */
static double W7(int a) { return a == 0 ? 0.25 : 0.125; }  /* 1/N_m, 1/(2N_m) */

/* index of the direction opposite to a */
static int opposite(const int (*E)[3], int q, int a)
{
    for (int b = 0; b < q; ++b)
        if (E[b][0] == -E[a][0] && E[b][1] == -E[a][1] && E[b][2] == -E[a][2])
            return b;
    return -1;
}

void orc_lattice_d3q19(int* E, double* w, int* opp)
{
    for (int a = 0; a < 19; ++a) {
        for (int d = 0; d < 3; ++d) E[a*3+d] = E19[a][d];
        w[a] = w19(a);
        opp[a] = opposite(E19, 19, a);
    }
}

/* ---------------------------------------------------------------------- */
/* Moment matrix T (Sec. 2; basis of App. A, D3Q19): each row is the      */
/* Gram-Schmidt polynomial of the particle velocity c = e_a named there.  */
/* ---------------------------------------------------------------------- */
static double T[19][19], Tinv[19][19];
static int tables_ready = 0;

static double row_poly(int k, const int* e)
{
    double cx = e[0], cy = e[1], cz = e[2];
    double c2 = cx*cx + cy*cy + cz*cz;
    switch (k) {
    case 0:  return 1.0;                                    /* rho    */
    case 1:  return 19.0*c2 - 30.0;                         /* e      */
    case 2:  return (21.0*c2*c2 - 53.0*c2 + 24.0) / 2.0;    /* e^2    */
    case 3:  return cx;                                     /* j_x    */
    case 4:  return (5.0*c2 - 9.0) * cx;                    /* q_x    */
    case 5:  return cy;                                     /* j_y    */
    case 6:  return (5.0*c2 - 9.0) * cy;                    /* q_y    */
    case 7:  return cz;                                     /* j_z    */
    case 8:  return (5.0*c2 - 9.0) * cz;                    /* q_z    */
    case 9:  return 3.0*cx*cx - c2;                         /* 3p_xx  */
    case 10: return (3.0*c2 - 5.0) * (3.0*cx*cx - c2);      /* 3pi_xx */
    case 11: return cy*cy - cz*cz;                          /* p_ww   */
    case 12: return (3.0*c2 - 5.0) * (cy*cy - cz*cz);       /* pi_ww  */
    case 13: return cx*cy;                                  /* p_xy   */
    case 14: return cy*cz;                                  /* p_yz   */
    case 15: return cx*cz;                                  /* p_xz   */
    case 16: return (cy*cy - cz*cz) * cx;                   /* m_x    */
    case 17: return (cz*cz - cx*cx) * cy;                   /* m_y    */
    case 18: return (cx*cx - cy*cy) * cz;                   /* m_z    */
    }
    return 0.0;
}

static void build_tables(void)
{
    if (tables_ready) return;
    double norm2[19];
    for (int k = 0; k < 19; ++k) {
        norm2[k] = 0.0;
        for (int a = 0; a < 19; ++a) {
            T[k][a] = row_poly(k, E19[a]);
            norm2[k] += T[k][a] * T[k][a];
        }
    }
    /* T^-1 = T^t diag(1/|row_k|^2) because the rows are mutually orthogonal */
    for (int a = 0; a < 19; ++a)
        for (int k = 0; k < 19; ++k)
            Tinv[a][k] = T[k][a] / norm2[k];
    tables_ready = 1;
}

void orc_moment_matrix(double* out)
{
    build_tables();
    for (int k = 0; k < 19; ++k) for (int a = 0; a < 19; ++a) out[k*19+a] = T[k][a];
}

void orc_inverse_moment_matrix(double* out)
{
    build_tables();
    for (int a = 0; a < 19; ++a) for (int k = 0; k < 19; ++k) out[a*19+k] = Tinv[a][k];
}

/* ---------------------------------------------------------------------- */
/* Preconditioned equilibrium moments f^eq,* (Sec. 3, D3Q19 list):        */
/* only the terms nonlinear in j carry 1/gamma.                           */
/* ---------------------------------------------------------------------- */
void orc_equilibrium_moments(double rho, const double* j, double gamma, double* meq)
{
    double jj = j[0]*j[0] + j[1]*j[1] + j[2]*j[2];
    double gr = gamma * rho;
    meq[0]  = rho;
    meq[1]  = -11.0*rho + 19.0*jj/gr;
    meq[2]  = 3.0*rho - (11.0/2.0)*jj/gr;
    meq[3]  = j[0];
    meq[4]  = -(2.0/3.0)*j[0];
    meq[5]  = j[1];
    meq[6]  = -(2.0/3.0)*j[1];
    meq[7]  = j[2];
    meq[8]  = -(2.0/3.0)*j[2];
    meq[9]  = (3.0*j[0]*j[0] - jj)/gr;
    meq[10] = -0.5*meq[9];                 /* 3 pi_xx = 3(-1/2 p_xx)        */
    meq[11] = (j[1]*j[1] - j[2]*j[2])/gr;
    meq[12] = -0.5*meq[11];                /* pi_ww = -1/2 p_ww             */
    meq[13] = j[0]*j[1]/gr;
    meq[14] = j[1]*j[2]/gr;
    meq[15] = j[0]*j[2]/gr;
    meq[16] = 0.0;
    meq[17] = 0.0;
    meq[18] = 0.0;
}

/* ---------------------------------------------------------------------- */
/* Moment projections of the source (App. A, D3Q19), then                  */
/* S^* = P_S S (Eq. precondsourceterm) with the D3Q19 diagonal P_S.        */
/* ---------------------------------------------------------------------- */
static void source_moments_unpreconditioned(const double* F, const double* u, double* S)
{
    double Fu = F[0]*u[0] + F[1]*u[1] + F[2]*u[2];
    S[0]  = 0.0;
    S[1]  = 38.0*Fu;
    S[2]  = -11.0*Fu;
    S[3]  = F[0];
    S[4]  = -(2.0/3.0)*F[0];
    S[5]  = F[1];
    S[6]  = -(2.0/3.0)*F[1];
    S[7]  = F[2];
    S[8]  = -(2.0/3.0)*F[2];
    S[9]  = 2.0*(2.0*F[0]*u[0] - F[1]*u[1] - F[2]*u[2]);
    S[10] = -(2.0*F[0]*u[0] - F[1]*u[1] - F[2]*u[2]);
    S[11] = 2.0*(F[1]*u[1] - F[2]*u[2]);
    S[12] = -(F[1]*u[1] - F[2]*u[2]);
    S[13] = F[0]*u[1] + F[1]*u[0];
    S[14] = F[1]*u[2] + F[2]*u[1];
    S[15] = F[0]*u[2] + F[2]*u[0];
    S[16] = 0.0;
    S[17] = 0.0;
    S[18] = 0.0;
}

void orc_source_precond_diag(double gamma, double* PS)
{
    double g1 = 1.0/gamma, g2 = 1.0/(gamma*gamma);
    PS[0] = 1.0; PS[1] = g2; PS[2] = g2;
    for (int k = 3; k <= 8; ++k) PS[k] = g1;
    for (int k = 9; k <= 15; ++k) PS[k] = g2;
    PS[16] = 1.0; PS[17] = 1.0; PS[18] = 1.0;
}

void orc_source_moments(const double* F, const double* u, double gamma, double* Sstar)
{
    double S[19], PS[19];
    source_moments_unpreconditioned(F, u, S);
    orc_source_precond_diag(gamma, PS);
    for (int k = 0; k < 19; ++k) Sstar[k] = PS[k] * S[k];
}

/* ---------------------------------------------------------------------- */
/* Relaxation rates Lambda^* (Sec. 3): 1/s_nu* = 3 nu/gamma + 1/2 on the   */
/* viscous rows 9, 11, 13, 14, 15; the other rows keep the given rates.   */
/* ---------------------------------------------------------------------- */
void orc_relaxation_rates(const orc_params* p, double* s)
{
    double snu = 1.0 / (3.0*p->nu/p->gamma + 0.5);
    for (int k = 0; k < 19; ++k) s[k] = p->s[k];
    s[9] = s[11] = s[13] = s[14] = s[15] = snu;
}

/* tau_m* = eta/(gamma_m theta_m) + 1/2 (Eq. mrelaxationtime) */
double orc_tau_m(const orc_params* p)
{
    return p->eta / (p->gamma_m * THETA_M) + 0.5;
}

/* ---------------------------------------------------------------------- */
/* Vector equilibrium with the low-Pr_m scaling (Sec. 4.1):                */
/* g^eq,*_aj = W_a { B_j + (e_ak/theta_m)(chi/gamma_m)(u_k B_j - B_k u_j) } */
/* stored as geq[j*7 + a].                                                */
/* ---------------------------------------------------------------------- */
void orc_vector_equilibrium(const orc_params* p, const double* u, const double* B, double* geq)
{
    double c = p->chi / p->gamma_m;
    for (int j = 0; j < 3; ++j)
        for (int a = 0; a < 7; ++a) {
            double conv = 0.0;
            for (int k = 0; k < 3; ++k)
                conv += E7[a][k] * (u[k]*B[j] - B[k]*u[j]);
            geq[j*7+a] = W7(a) * (B[j] + conv * c / THETA_M);
        }
}

static int levi_civita(int i, int j, int k)
{
    if (i == j || j == k || i == k) return 0;
    if ((i == 0 && j == 1 && k == 2) || (i == 1 && j == 2 && k == 0) || (i == 2 && j == 0 && k == 1))
        return 1;
    return -1;
}

/* J_i = (1/(mu chi)) (curl B)_i from the non-equilibrium first moment of g
 * (Sec. 4.1 with the index order of App. C; see the header). */
void orc_current_density(const orc_params* p, const double* g, const double* geq, double* J)
{
    double Lneq[3][3];
    for (int a2 = 0; a2 < 3; ++a2)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int a = 0; a < 7; ++a)
                s += E7[a][a2] * (g[b*7+a] - geq[b*7+a]);
            Lneq[a2][b] = s;
        }
    double coef = -1.0 / (p->mu * p->chi * orc_tau_m(p) * THETA_M);
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                s += levi_civita(i, j, k) * Lneq[j][k];
        J[i] = coef * s;
    }
}

/* ---------------------------------------------------------------------- */
/* One node: macroscopic fields, coupling, collision (Eqs. ppostcollision, */
/* prelax_term, precondhydrofields, mcollision).                           */
/* ---------------------------------------------------------------------- */
typedef struct {
    double rho, u[3], B[3], FL[3], F[3];
} node_macro;

static void node_collide(const orc_params* p, const double* s, double tau_m,
                         const double* f, const double* g, const double* FLprev,
                         const double* Fext, double* ftilde, double* gtilde,
                         node_macro* out)
{
    const double gam = p->gamma;
    /* rho and the bare first moment m = sum f e */
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 19; ++a) {
        rho += f[a];
        for (int d = 0; d < 3; ++d) m[d] += f[a] * E19[a][d];
    }
    double F[3], FL[3] = {0.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 0.0};
    double geq[21];
    if (p->induction) {
        /* B_i = sum_a g_ai (Eq. magneticinduction) */
        for (int j = 0; j < 3; ++j)
            for (int a = 0; a < 7; ++a) B[j] += g[j*7+a];
        /* velocity with the previous step's Lorentz force in the half-force */
        double u0[3];
        for (int d = 0; d < 3; ++d)
            u0[d] = (m[d] + 0.5*(Fext[d] + FLprev[d])/gam) / rho;
        orc_vector_equilibrium(p, u0, B, geq);
        double J[3];
        orc_current_density(p, g, geq, J);
        /* F_Lorentz = J x B */
        FL[0] = J[1]*B[2] - J[2]*B[1];
        FL[1] = J[2]*B[0] - J[0]*B[2];
        FL[2] = J[0]*B[1] - J[1]*B[0];
    }
    for (int d = 0; d < 3; ++d) F[d] = Fext[d] + FL[d];
    /* j = sum f e + F/(2 gamma), u = j / rho (Eq. precondhydrofields) */
    double jv[3], u[3];
    for (int d = 0; d < 3; ++d) { jv[d] = m[d] + 0.5*F[d]/gam; u[d] = jv[d]/rho; }

    /* moments f^ = T f */
    double fh[19];
    for (int k = 0; k < 19; ++k) {
        double acc = 0.0;
        for (int a = 0; a < 19; ++a) acc += T[k][a] * f[a];
        fh[k] = acc;
    }
    double meq[19], Ss[19];
    orc_equilibrium_moments(rho, jv, gam, meq);
    orc_source_moments(F, u, gam, Ss);
    /* -Lambda* (f^ - f^eq*) + (I - Lambda*  / 2) S*  (Eq. prelax_term) */
    double dm[19];
    for (int k = 0; k < 19; ++k)
        dm[k] = -s[k]*(fh[k] - meq[k]) + (1.0 - 0.5*s[k])*Ss[k];
    /* f~ = f + T^-1 [ ... ] */
    for (int a = 0; a < 19; ++a) {
        double acc = 0.0;
        for (int k = 0; k < 19; ++k) acc += Tinv[a][k] * dm[k];
        ftilde[a] = f[a] + acc;
    }
    if (p->induction) {
        for (int i = 0; i < 21; ++i)
            gtilde[i] = g[i] - (g[i] - geq[i]) / tau_m;
    }
    if (out) {
        out->rho = rho;
        for (int d = 0; d < 3; ++d) {
            out->u[d] = u[d]; out->B[d] = B[d]; out->FL[d] = FL[d]; out->F[d] = F[d];
        }
    }
}

/* single-node collision, exposed for the moment-space pins */
void orc_collide_node(const orc_params* p, const double* f, const double* g,
                      const double* FLprev, const double* Fext,
                      double* ftilde, double* gtilde, double* macro /* rho,u3,B3,FL3 */)
{
    build_tables();
    double s[19];
    orc_relaxation_rates(p, s);
    double z3[3] = {0.0, 0.0, 0.0};
    node_macro nm;
    node_collide(p, s, p->induction ? orc_tau_m(p) : 1.0, f, g,
                 FLprev ? FLprev : z3, Fext ? Fext : z3, ftilde, gtilde, &nm);
    if (macro) {
        macro[0] = nm.rho;
        for (int d = 0; d < 3; ++d) {
            macro[1+d] = nm.u[d]; macro[4+d] = nm.B[d]; macro[7+d] = nm.FL[d];
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Geometry: a node is solid when it lies on a wall plane.                 */
/* ---------------------------------------------------------------------- */
static int is_solid(const orc_params* p, int x, int y, int z)
{
    int c[3] = {x, y, z};
    int n[3] = {p->nx, p->ny, p->nz};
    for (int d = 0; d < 3; ++d) {
        if (p->wall_lo[d] && c[d] == 0) return 1;
        if (p->wall_hi[d] && c[d] == n[d]-1) return 1;
    }
    return 0;
}

static int wrap(int c, int n) { c %= n; return c < 0 ? c + n : c; }

int orc_is_solid(const orc_params* p, int x, int y, int z) { return is_solid(p, x, y, z); }

/* Solid for the flow lattice: a wall plane, or outside the fluid box. */
static int flow_solid(const orc_params* p, int x, int y, int z)
{
    if (is_solid(p, x, y, z)) return 1;
    if (!p->box) return 0;
    int c[3] = {x, y, z};
    for (int d = 0; d < 3; ++d)
        if (c[d] < p->box_lo[d] || c[d] > p->box_hi[d]) return 1;
    return 0;
}

int orc_flow_solid(const orc_params* p, int x, int y, int z) { return flow_solid(p, x, y, z); }

/* Highest fluid z plane of the flow lattice (the lid lies above it). */
static int top_fluid_z(const orc_params* p)
{
    if (p->box) return p->box_hi[2];
    return p->wall_hi[2] ? p->nz - 2 : p->nz - 1;
}

/* ---------------------------------------------------------------------- */
/* Initial state: rest equilibrium f = w rho0, g = W B0, F_L = 0.          */
/* ---------------------------------------------------------------------- */
void orc_init_state(const orc_params* p, double* f, double* g, double* FL)
{
    long N = (long)p->nx * p->ny * p->nz;
    for (long n = 0; n < N; ++n) {
        for (int a = 0; a < 19; ++a) f[n*19+a] = w19(a) * p->rho0;
        if (g) for (int j = 0; j < 3; ++j) for (int a = 0; a < 7; ++a) g[n*21+j*7+a] = W7(a) * p->B0[j];
        if (FL) for (int d = 0; d < 3; ++d) FL[n*3+d] = 0.0;
    }
}

static void node_force(const orc_params* p, const double* Fext, long n, double* F)
{
    for (int d = 0; d < 3; ++d) F[d] = p->F[d] + (Fext ? Fext[n*3+d] : 0.0);
}

/* ---------------------------------------------------------------------- */
/* Macroscopic fields of the current state (rho, u, B, and the Lorentz     */
/* force that the next collision would form), without changing the state. */
/* ---------------------------------------------------------------------- */
void orc_fields(const orc_params* p, const double* f, const double* g, const double* FL,
                const double* Fext, double* rho, double* u, double* B, double* FLnew)
{
    build_tables();
    double s[19];
    orc_relaxation_rates(p, s);
    double tau_m = p->induction ? orc_tau_m(p) : 1.0;
    long N = (long)p->nx * p->ny * p->nz;
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        int x = (int)(n % p->nx), y = (int)((n / p->nx) % p->ny), z = (int)(n / ((long)p->nx*p->ny));
        if (flow_solid(p, x, y, z)) {
            if (rho) rho[n] = 0.0;
            for (int d = 0; d < 3; ++d) {
                if (u) u[n*3+d] = 0.0;
                if (B) B[n*3+d] = 0.0;
                if (FLnew) FLnew[n*3+d] = 0.0;
            }
            /* outside the fluid box the vector lattice still carries B */
            if (B && p->induction && !is_solid(p, x, y, z))
                for (int j = 0; j < 3; ++j) {
                    double b = 0.0;
                    for (int a = 0; a < 7; ++a) b += g[n*21+j*7+a];
                    B[n*3+j] = b;
                }
            continue;
        }
        double ft[19], gt[21], Fn[3], z3[3] = {0.0, 0.0, 0.0};
        node_force(p, Fext, n, Fn);
        node_macro nm;
        node_collide(p, s, tau_m, f + n*19, p->induction ? g + n*21 : NULL,
                     p->induction ? FL + n*3 : z3, Fn, ft, gt, &nm);
        if (rho) rho[n] = nm.rho;
        for (int d = 0; d < 3; ++d) {
            if (u) u[n*3+d] = nm.u[d];
            if (B) B[n*3+d] = nm.B[d];
            if (FLnew) FLnew[n*3+d] = nm.FL[d];
        }
    }
}

/* ---------------------------------------------------------------------- */
/* One time step: collide every fluid node, then stream (push) with       */
/* half-way bounce-back for f and anti-bounce-back for g at solid links.   */
/* fn, gn are output buffers of the same size as f, g.                     */
/* ---------------------------------------------------------------------- */
static void step(const orc_params* p, const double* s, double tau_m,
                 const double* f, const double* g, double* FL, const double* Fext,
                 double* fn, double* gn, double* uout)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long N = (long)nx * ny * nz;
    static int opp19[19], opp7[7];
    static int opp_ready = 0;
    if (!opp_ready) {
        for (int a = 0; a < 19; ++a) opp19[a] = opposite(E19, 19, a);
        for (int a = 0; a < 7; ++a) opp7[a] = opposite(E7, 7, a);
        opp_ready = 1;
    }
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx*ny));
        if (is_solid(p, x, y, z)) continue;
        const int fluid = !flow_solid(p, x, y, z);
        double ft[19], gt[21], Fn[3], z3[3] = {0.0, 0.0, 0.0};
        if (fluid) {
            node_force(p, Fext, n, Fn);
            node_macro nm;
            node_collide(p, s, tau_m, f + n*19, p->induction ? g + n*21 : NULL,
                         p->induction ? FL + n*3 : z3, Fn, ft, gt, &nm);
            if (uout) for (int d = 0; d < 3; ++d) uout[n*3+d] = nm.u[d];
            if (p->induction) for (int d = 0; d < 3; ++d) FL[n*3+d] = nm.FL[d];
        } else {
            if (!p->induction) continue;
            /* outside the fluid box: the vector lattice alone, with u = 0
               (Eq. mcollision, g^eq of B only) and no Lorentz force */
            double B[3] = {0.0, 0.0, 0.0}, geq[21];
            for (int j = 0; j < 3; ++j)
                for (int a = 0; a < 7; ++a) B[j] += g[n*21+j*7+a];
            orc_vector_equilibrium(p, z3, B, geq);
            for (int i = 0; i < 21; ++i) gt[i] = g[n*21+i] - (g[n*21+i] - geq[i]) / tau_m;
            for (int d = 0; d < 3; ++d) FL[n*3+d] = 0.0;
            if (uout) for (int d = 0; d < 3; ++d) uout[n*3+d] = 0.0;
        }
        /* streaming, Eq. pstreaming: f_a(x + e_a, t+1) = f~_a(x, t); a link
           into the flow boundary is bounced back half-way, with the lid's
           momentum when it ends above the highest fluid z plane */
        if (fluid) {
            const int top = top_fluid_z(p);
            for (int a = 0; a < 19; ++a) {
                int xt = wrap(x + E19[a][0], nx), yt = wrap(y + E19[a][1], ny), zt = wrap(z + E19[a][2], nz);
                if (flow_solid(p, xt, yt, zt)) {
                    double wall = 0.0;
                    if (z + E19[a][2] > top) {
                        double eU = E19[a][0]*p->U_lid[0] + E19[a][1]*p->U_lid[1] + E19[a][2]*p->U_lid[2];
                        wall = 6.0 * w19(a) * p->rho0 * eU;
                    }
                    fn[n*19 + opp19[a]] = ft[a] - wall;
                } else {
                    fn[(((long)zt*ny + yt)*nx + xt)*19 + a] = ft[a];
                }
            }
        }
        if (p->induction) {
            /* Eq. mstreaming on D3Q7, anti-bounce-back at insulating walls */
            for (int a = 0; a < 7; ++a) {
                int xt = wrap(x + E7[a][0], nx), yt = wrap(y + E7[a][1], ny), zt = wrap(z + E7[a][2], nz);
                int solid = is_solid(p, xt, yt, zt);
                long tn = (((long)zt*ny + yt)*nx + xt);
                for (int j = 0; j < 3; ++j) {
                    if (solid)
                        gn[n*21 + j*7 + opp7[a]] = -gt[j*7+a] + 2.0*W7(a)*p->B0[j];
                    else
                        gn[tn*21 + j*7 + a] = gt[j*7+a];
                }
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Time march with the steady-state residual (Sec. 5):                     */
/* r(t) = ||u(t) - u(t-10)||_2 / ||u(t)||_2, t = 10, 20, ...               */
/*                                                                         */
/* State (f, g, FL) is at time level t0 on entry and at the returned level */
/* on exit.  usnap (3N) holds u at level *tsnap (-1: no snapshot yet); at  */
/* every level t that is a multiple of 10 and differs from *tsnap the      */
/* residual against the snapshot is recorded (when a snapshot exists) and  */
/* the snapshot is replaced by u(t).  hist receives rows                   */
/* (t, r, num, den, mass, Mx, My, Mz) with M the fluid momentum sum at t.  */
/* Returns the level reached: the first t with r(t) <= tol (tol > 0) or a  */
/* non-finite r, else t0 + nsteps.                                         */
/* ---------------------------------------------------------------------- */
long orc_run(const orc_params* p, double* f, double* g, double* FL, const double* Fext,
             double* usnap, long* tsnap, long t0, long nsteps, double tol,
             double* hist, long hist_cap, long* nhist)
{
    build_tables();
    double s[19];
    orc_relaxation_rates(p, s);
    double tau_m = p->induction ? orc_tau_m(p) : 1.0;
    const long N = (long)p->nx * p->ny * p->nz;
    double* fn = (double*)malloc(sizeof(double) * 19 * N);
    double* gn = p->induction ? (double*)malloc(sizeof(double) * 21 * N) : NULL;
    double* ut = (double*)malloc(sizeof(double) * 3 * N);
    double* rh = (double*)malloc(sizeof(double) * N);
    long nh = nhist ? *nhist : 0;
    long t = t0;
    /* solid nodes are never written by the step; keep their contents */
    memcpy(fn, f, sizeof(double) * 19 * N);
    if (gn) memcpy(gn, g, sizeof(double) * 21 * N);
    for (; t < t0 + nsteps; ++t) {
        if (t % 10 == 0 && t != *tsnap) {
            orc_fields(p, f, g, FL, Fext, rh, ut, NULL, NULL);
            int stop = 0;
            if (*tsnap >= 0) {
                double num = 0.0, den = 0.0, mass = 0.0, mom[3] = {0.0, 0.0, 0.0};
                for (long n = 0; n < N; ++n) {
                    int x = (int)(n % p->nx), y = (int)((n / p->nx) % p->ny), z = (int)(n / ((long)p->nx*p->ny));
                    if (flow_solid(p, x, y, z)) continue;
                    for (int d = 0; d < 3; ++d) {
                        double du = ut[n*3+d] - usnap[n*3+d];
                        num += du*du;
                        den += ut[n*3+d]*ut[n*3+d];
                        mom[d] += rh[n]*ut[n*3+d];
                    }
                    mass += rh[n];
                }
                double r = den > 0.0 ? sqrt(num/den) : (num > 0.0 ? INFINITY : 0.0);
                if (!isfinite(num) || !isfinite(den)) r = NAN;   /* a diverged state is never "converged" */
                if (hist && nh < hist_cap) {
                    double* h = hist + nh*8;
                    h[0] = (double)t; h[1] = r; h[2] = num; h[3] = den; h[4] = mass;
                    h[5] = mom[0]; h[6] = mom[1]; h[7] = mom[2];
                    ++nh;
                }
                stop = (tol > 0.0 && r <= tol) || !isfinite(r);
            }
            memcpy(usnap, ut, sizeof(double) * 3 * N);
            *tsnap = t;
            if (stop) break;
        }
        step(p, s, tau_m, f, g, FL, Fext, fn, gn, NULL);
        memcpy(f, fn, sizeof(double) * 19 * N);
        if (gn) memcpy(g, gn, sizeof(double) * 21 * N);
    }
    if (nhist) *nhist = nh;
    free(fn); free(gn); free(ut); free(rh);
    return t;
}

/* ---------------------------------------------------------------------- */
/* Node Jacobians for the gradient checks.  The paper has no adjoint: the  */
/* derivative of the node update above is taken numerically, by central    */
/* differences of the unchanged node_collide in FP64.                      */
/*   inputs  x = (f[19], g[21], F_L of the previous step[3], F_ext[3])     */
/*   outputs y = (f~[19], g~[21], F_L[3], u[3])                            */
/* J[i*46 + k] = dy_i/dx_k with step h[k] for input k.  Without induction  */
/* the g and F_L columns and rows are zero.                                */
/* ---------------------------------------------------------------------- */
#define ORC_NJ 46

static void node_outputs(const orc_params* p, const double* s, double tau_m, const double* x, double* y)
{
    double ft[19], gt[21];
    node_macro nm;
    node_collide(p, s, tau_m, x, p->induction ? x + 19 : NULL, x + 40, x + 43, ft, gt, &nm);
    for (int i = 0; i < ORC_NJ; ++i) y[i] = 0.0;
    for (int a = 0; a < 19; ++a) y[a] = ft[a];
    if (p->induction) {
        for (int i = 0; i < 21; ++i) y[19 + i] = gt[i];
        for (int d = 0; d < 3; ++d) y[40 + d] = nm.FL[d];
    }
    for (int d = 0; d < 3; ++d) y[43 + d] = nm.u[d];
}

static void node_jacobian(const orc_params* p, const double* s, double tau_m, const double* x0,
                          const double* h, double* J)
{
    double x[ORC_NJ], yp[ORC_NJ], ym[ORC_NJ];
    for (int i = 0; i < ORC_NJ * ORC_NJ; ++i) J[i] = 0.0;
    for (int k = 0; k < ORC_NJ; ++k) {
        if (!p->induction && k >= 19 && k < 43) continue;
        for (int i = 0; i < ORC_NJ; ++i) x[i] = x0[i];
        x[k] = x0[k] + h[k];
        node_outputs(p, s, tau_m, x, yp);
        x[k] = x0[k] - h[k];
        node_outputs(p, s, tau_m, x, ym);
        for (int i = 0; i < ORC_NJ; ++i) J[i*ORC_NJ + k] = (yp[i] - ym[i]) / (2.0 * h[k]);
    }
}

/* One node: f[19], g[21] (may be NULL without induction), FLprev[3],
 * Fext[3] (the node's total external force). */
void orc_node_jacobian(const orc_params* p, const double* f, const double* g, const double* FLprev,
                       const double* Fext, const double* h, double* J)
{
    build_tables();
    double s[19];
    orc_relaxation_rates(p, s);
    double tau_m = p->induction ? orc_tau_m(p) : 1.0;
    double x[ORC_NJ] = {0.0};
    for (int a = 0; a < 19; ++a) x[a] = f[a];
    if (p->induction) {
        for (int i = 0; i < 21; ++i) x[19 + i] = g[i];
        for (int d = 0; d < 3; ++d) x[40 + d] = FLprev[d];
    }
    for (int d = 0; d < 3; ++d) x[43 + d] = Fext[d];
    node_jacobian(p, s, tau_m, x, h, J);
}

/* Every node of a state (f, g, FL as in orc_run; Fext the [N][3] field or
 * NULL): J[n][46][46]; zero for solid nodes. */
void orc_state_jacobians(const orc_params* p, const double* f, const double* g, const double* FL,
                         const double* Fext, const double* h, double* J)
{
    build_tables();
    double s[19];
    orc_relaxation_rates(p, s);
    double tau_m = p->induction ? orc_tau_m(p) : 1.0;
    const long N = (long)p->nx * p->ny * p->nz;
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double* Jn = J + n * ORC_NJ * ORC_NJ;
        int x = (int)(n % p->nx), y = (int)((n / p->nx) % p->ny), z = (int)(n / ((long)p->nx*p->ny));
        if (is_solid(p, x, y, z)) {
            for (int i = 0; i < ORC_NJ * ORC_NJ; ++i) Jn[i] = 0.0;
            continue;
        }
        double xv[ORC_NJ] = {0.0}, Fn[3];
        for (int a = 0; a < 19; ++a) xv[a] = f[n*19 + a];
        if (p->induction) {
            for (int i = 0; i < 21; ++i) xv[19 + i] = g[n*21 + i];
            for (int d = 0; d < 3; ++d) xv[40 + d] = FL[n*3 + d];
        }
        node_force(p, Fext, n, Fn);
        for (int d = 0; d < 3; ++d) xv[43 + d] = Fn[d];
        node_jacobian(p, s, tau_m, xv, h, Jn);
    }
}

/* ---------------------------------------------------------------------- */
/* Threads (the CPU baseline uses every host core; results do not depend   */
/* on the thread count because every node is computed independently).     */
/* ---------------------------------------------------------------------- */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
