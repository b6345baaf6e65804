/*
 * glbe_oracle2d.c -- plain FP64 CPU oracle of the two-dimensional forms of
 * the preconditioned GLBE with forcing term (D2Q9, multiple relaxation times)
 * and of the preconditioned vector lattice kinetic equation for the magnetic
 * induction (D2Q5), arXiv:0809.4730 Secs. 2-4 and App. A (D2Q9 tables).
 *
 * TEST INFRASTRUCTURE ONLY, like glbe_oracle.c: only the test-suite, the
 * smoke check and the CPU baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Same design rules as the 3D oracle: IEEE FP64, fixed loop order, no FMA
 * contraction; the moment matrix is built from its defining polynomials and
 * applied as a dense 9x9 product, its inverse is T^t D^-1; storage is
 * array-of-structures f[n*9+a], g[n*10 + j*5 + a] (j = x, y), FL[n*2+i];
 * streaming is a push with half-way bounce-back (f) and anti-bounce-back to
 * B0 (g) at solid links.
 *
 * Readings (where the paper is silent):
 *   - D2Q9 ordering (Eq. velocityd2q9 gives the groups): 0 (0,0); 1 (1,0),
 *     2 (0,1), 3 (-1,0), 4 (0,-1); 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1);
 *     weights 4/9, 1/9, 1/36.
 *   - Moment basis (App. A, D2Q9 of the cited Gram-Schmidt construction):
 *     rho = 1, e = -4 + 3 c^2, e^2 = 4 - 21/2 c^2 + 9/2 c^4, j = c,
 *     q = (3 c^2 - 5) c, p_xx = c_x^2 - c_y^2, p_xy = c_x c_y; the App. A
 *     equilibrium and source tables fix this normalisation.
 *   - Rates (Sec. 3): s_7 = s_8 = s_nu* with 1/s_nu* = 3 nu/gamma + 1/2; the
 *     kinetic rates s_1 = 1.63, s_2 = 1.14, s_4 = s_6 = 1.92 (s_1 is printed
 *     both as the bulk-viscosity rate and as a kinetic rate; the kinetic
 *     value is taken, as for D3Q19); conserved rows 0, 3, 5 cannot matter.
 *   - D2Q5 (Sec. 4): 0 (0,0), 1 (1,0), 2 (-1,0), 3 (0,1), 4 (0,-1);
 *     N_m = 3, W_0 = 1/3, W_a = 1/6, theta_m = 1/3; B and u in the plane,
 *     J = J_z e_z with J_z = (1/(mu chi)) (d_x B_y - d_y B_x) from the
 *     non-equilibrium first moment (the index order of the 3D reading),
 *     Lorentz force J x B = (-J_z B_y, J_z B_x); the previous step's Lorentz
 *     force in the velocity of g^eq, as in 3D.
 */
#include <math.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>

typedef struct {
    int nx, ny;
    int wall_lo[2], wall_hi[2];  /* 1: the line at index 0 / n-1 is solid */
    double rho0, gamma, nu;
    double s[9];                 /* rates of the non-viscous rows; rows 7, 8 overwritten by s_nu* */
    double F[2];                 /* uniform force, added to the field */
    int induction;
    double gamma_m, eta, chi, mu;
    double B0[2];
} orc2_params;

int orc2_params_size(void) { return (int)sizeof(orc2_params); }

static const int E9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
static const int E5[5][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}};

static double w9(int a)
{
    int c2 = E9[a][0]*E9[a][0] + E9[a][1]*E9[a][1];
    return c2 == 0 ? 4.0/9.0 : (c2 == 1 ? 1.0/9.0 : 1.0/36.0);
}
static double W5(int a) { return a == 0 ? 1.0/3.0 : 1.0/6.0; }   /* 1/N_m, 1/(2 N_m), N_m = 3 */
static const double THETA2 = 1.0/3.0;

static int opp9(int a)
{
    for (int b = 0; b < 9; ++b)
        if (E9[b][0] == -E9[a][0] && E9[b][1] == -E9[a][1]) return b;
    return -1;
}
static int opp5(int a)
{
    for (int b = 0; b < 5; ++b)
        if (E5[b][0] == -E5[a][0] && E5[b][1] == -E5[a][1]) return b;
    return -1;
}

/* Row k of the moment matrix at velocity c (App. A, D2Q9). */
static double row2(int k, const int* c)
{
    const double cx = c[0], cy = c[1], c2 = cx*cx + cy*cy;
    switch (k) {
    case 0: return 1.0;
    case 1: return -4.0 + 3.0*c2;
    case 2: return 4.0 - 10.5*c2 + 4.5*c2*c2;
    case 3: return cx;
    case 4: return (3.0*c2 - 5.0)*cx;
    case 5: return cy;
    case 6: return (3.0*c2 - 5.0)*cy;
    case 7: return cx*cx - cy*cy;
    default: return cx*cy;
    }
}

static double T2[9][9], T2inv[9][9];
static int t2_ready = 0;

static void build2(void)
{
    if (t2_ready) return;
    for (int k = 0; k < 9; ++k)
        for (int a = 0; a < 9; ++a) T2[k][a] = row2(k, E9[a]);
    for (int k = 0; k < 9; ++k) {
        double nrm = 0.0;
        for (int a = 0; a < 9; ++a) nrm += T2[k][a]*T2[k][a];
        for (int a = 0; a < 9; ++a) T2inv[a][k] = T2[k][a]/nrm;
    }
    t2_ready = 1;
}

void orc2_moment_matrix(double* out)
{
    build2();
    for (int k = 0; k < 9; ++k) for (int a = 0; a < 9; ++a) out[k*9+a] = T2[k][a];
}

void orc2_lattice(int* E, double* w, int* opp)
{
    for (int a = 0; a < 9; ++a) {
        E[a*2] = E9[a][0]; E[a*2+1] = E9[a][1];
        w[a] = w9(a);
        opp[a] = opp9(a);
    }
}

/* Preconditioned equilibrium moments (Sec. 3, D2Q9). */
void orc2_equilibrium_moments(double rho, const double* j, double gamma, double* meq)
{
    const double jj = j[0]*j[0] + j[1]*j[1];
    meq[0] = rho;
    meq[1] = -2.0*rho + 3.0*jj/(gamma*rho);
    meq[2] = rho - 3.0*jj/(gamma*rho);
    meq[3] = j[0];
    meq[4] = -j[0];
    meq[5] = j[1];
    meq[6] = -j[1];
    meq[7] = (j[0]*j[0] - j[1]*j[1])/(gamma*rho);
    meq[8] = j[0]*j[1]/(gamma*rho);
}

/* P_S = diag(1, 1/g^2, 1/g^2, 1/g, 1/g, 1/g, 1/g, 1/g^2, 1/g^2), Eq. precondsourceterm (D2Q9). */
void orc2_source_precond_diag(double gamma, double* PS)
{
    const double ig = 1.0/gamma, ig2 = ig*ig;
    const double d[9] = {1.0, ig2, ig2, ig, ig, ig, ig, ig2, ig2};
    for (int k = 0; k < 9; ++k) PS[k] = d[k];
}

/* Preconditioned source moments S* = P_S S (App. A table of S, D2Q9). */
void orc2_source_moments(const double* F, const double* u, double gamma, double* Ss)
{
    const double Fu = F[0]*u[0] + F[1]*u[1];
    double S[9];
    S[0] = 0.0;
    S[1] = 6.0*Fu;
    S[2] = -6.0*Fu;
    S[3] = F[0];
    S[4] = -F[0];
    S[5] = F[1];
    S[6] = -F[1];
    S[7] = 2.0*(F[0]*u[0] - F[1]*u[1]);
    S[8] = F[0]*u[1] + F[1]*u[0];
    double PS[9];
    orc2_source_precond_diag(gamma, PS);
    for (int k = 0; k < 9; ++k) Ss[k] = PS[k]*S[k];
}

void orc2_relaxation_rates(const orc2_params* p, double* s)
{
    for (int k = 0; k < 9; ++k) s[k] = p->s[k];
    const double snu = 1.0/(3.0*p->nu/p->gamma + 0.5);
    s[7] = s[8] = snu;
}

double orc2_tau_m(const orc2_params* p) { return p->eta/(p->gamma_m*THETA2) + 0.5; }

/* g^eq,*_ja = W_a [B_j + e_ak (chi/gamma_m)(u_k B_j - B_k u_j)/theta_m], Eq.
   mageqmoment with the low-Pr_m scaling of Sec. 4.1; out[j*5+a]. */
void orc2_vector_equilibrium(const orc2_params* p, const double* u, const double* B, double* geq)
{
    for (int j = 0; j < 2; ++j)
        for (int a = 0; a < 5; ++a) {
            double conv = 0.0;
            for (int k = 0; k < 2; ++k)
                conv += E5[a][k]*(u[k]*B[j] - B[k]*u[j]);
            geq[j*5+a] = W5(a)*(B[j] + conv*(p->chi/p->gamma_m)/THETA2);
        }
}

/* J_z = -(1/(mu chi tau_m theta_m)) (Lneq_xy - Lneq_yx), Lneq_jk = sum_a e_aj (g - g^eq)_ak */
static double current_z(const orc2_params* p, const double* g, const double* geq)
{
    double L[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int jj = 0; jj < 2; ++jj)
        for (int k = 0; k < 2; ++k)
            for (int a = 0; a < 5; ++a) L[jj][k] += E5[a][jj]*(g[k*5+a] - geq[k*5+a]);
    const double c = 1.0/(p->mu*p->chi*orc2_tau_m(p)*THETA2);
    return -c*(L[0][1] - L[1][0]);
}

double orc2_current_z(const orc2_params* p, const double* g, const double* geq) { return current_z(p, g, geq); }

typedef struct { double rho, u[2], B[2], FL[2]; } node2_macro;

static void node2_collide(const orc2_params* p, const double* s, double tau_m, const double* f, const double* g,
                          const double* FLprev, const double* Fext, double* ft, double* gt, node2_macro* out)
{
    const double gam = p->gamma;
    double rho = 0.0, m[2] = {0.0, 0.0};
    for (int a = 0; a < 9; ++a) {
        rho += f[a];
        for (int d = 0; d < 2; ++d) m[d] += f[a]*E9[a][d];
    }
    double FL[2] = {0.0, 0.0}, B[2] = {0.0, 0.0}, geq[10];
    if (p->induction) {
        for (int j = 0; j < 2; ++j)
            for (int a = 0; a < 5; ++a) B[j] += g[j*5+a];
        double u0[2];
        for (int d = 0; d < 2; ++d) u0[d] = (m[d] + 0.5*(Fext[d] + FLprev[d])/gam)/rho;
        orc2_vector_equilibrium(p, u0, B, geq);
        const double Jz = current_z(p, g, geq);
        FL[0] = -Jz*B[1];
        FL[1] = Jz*B[0];
    }
    double F[2], jv[2], u[2];
    for (int d = 0; d < 2; ++d) {
        F[d] = Fext[d] + FL[d];
        jv[d] = m[d] + 0.5*F[d]/gam;
        u[d] = jv[d]/rho;
    }
    double fh[9], meq[9], Ss[9], dm[9];
    for (int k = 0; k < 9; ++k) {
        double acc = 0.0;
        for (int a = 0; a < 9; ++a) acc += T2[k][a]*f[a];
        fh[k] = acc;
    }
    orc2_equilibrium_moments(rho, jv, gam, meq);
    orc2_source_moments(F, u, gam, Ss);
    for (int k = 0; k < 9; ++k) dm[k] = -s[k]*(fh[k] - meq[k]) + (1.0 - 0.5*s[k])*Ss[k];
    for (int a = 0; a < 9; ++a) {
        double acc = 0.0;
        for (int k = 0; k < 9; ++k) acc += T2inv[a][k]*dm[k];
        ft[a] = f[a] + acc;
    }
    if (p->induction)
        for (int i = 0; i < 10; ++i) gt[i] = g[i] - (g[i] - geq[i])/tau_m;
    if (out) {
        out->rho = rho;
        for (int d = 0; d < 2; ++d) { out->u[d] = u[d]; out->B[d] = B[d]; out->FL[d] = FL[d]; }
    }
}

/* One node's collision (test access): mac = (rho, u[2], B[2], FL[2]). */
void orc2_collide_node(const orc2_params* p, const double* f, const double* g, const double* FLprev,
                       const double* Fext, double* ft, double* gt, double* mac)
{
    build2();
    double s[9], z2[2] = {0.0, 0.0};
    orc2_relaxation_rates(p, s);
    const double tau_m = p->induction ? orc2_tau_m(p) : 1.0;
    double Fn[2];
    for (int d = 0; d < 2; ++d) Fn[d] = p->F[d] + (Fext ? Fext[d] : 0.0);
    node2_macro nm;
    node2_collide(p, s, tau_m, f, p->induction ? g : NULL, (p->induction && FLprev) ? FLprev : z2, Fn, ft, gt, &nm);
    mac[0] = nm.rho;
    for (int d = 0; d < 2; ++d) { mac[1+d] = nm.u[d]; mac[3+d] = nm.B[d]; mac[5+d] = nm.FL[d]; }
}

static int solid2(const orc2_params* p, int x, int y)
{
    return (p->wall_lo[0] && x == 0) || (p->wall_hi[0] && x == p->nx - 1) ||
           (p->wall_lo[1] && y == 0) || (p->wall_hi[1] && y == p->ny - 1);
}
int orc2_is_solid(const orc2_params* p, int x, int y) { return solid2(p, x, y); }
static int wrap2(int c, int n) { c %= n; return c < 0 ? c + n : c; }

void orc2_init_state(const orc2_params* p, double* f, double* g, double* FL)
{
    const long N = (long)p->nx*p->ny;
    for (long n = 0; n < N; ++n) {
        for (int a = 0; a < 9; ++a) f[n*9+a] = w9(a)*p->rho0;
        if (g) for (int j = 0; j < 2; ++j) for (int a = 0; a < 5; ++a) g[n*10+j*5+a] = W5(a)*p->B0[j];
        if (FL) FL[n*2] = FL[n*2+1] = 0.0;
    }
}

void orc2_fields(const orc2_params* p, const double* f, const double* g, const double* FL, const double* Fext,
                 double* rho, double* u, double* B)
{
    build2();
    double s[9];
    orc2_relaxation_rates(p, s);
    const double tau_m = p->induction ? orc2_tau_m(p) : 1.0;
    const long N = (long)p->nx*p->ny;
    for (long n = 0; n < N; ++n) {
        const int x = (int)(n % p->nx), y = (int)(n / p->nx);
        if (solid2(p, x, y)) {
            if (rho) rho[n] = 0.0;
            for (int d = 0; d < 2; ++d) { if (u) u[n*2+d] = 0.0; if (B) B[n*2+d] = 0.0; }
            continue;
        }
        double ft[9], gt[10], Fn[2], z2[2] = {0.0, 0.0};
        for (int d = 0; d < 2; ++d) Fn[d] = p->F[d] + (Fext ? Fext[n*2+d] : 0.0);
        node2_macro nm;
        node2_collide(p, s, tau_m, f + n*9, p->induction ? g + n*10 : NULL, p->induction ? FL + n*2 : z2, Fn,
                      ft, gt, &nm);
        if (rho) rho[n] = nm.rho;
        for (int d = 0; d < 2; ++d) { if (u) u[n*2+d] = nm.u[d]; if (B) B[n*2+d] = nm.B[d]; }
    }
}

static void step2(const orc2_params* p, const double* s, double tau_m, const double* f, const double* g, double* FL,
                  const double* Fext, double* fn, double* gn)
{
    const int nx = p->nx, ny = p->ny;
    const long N = (long)nx*ny;
    /* every target slot is written by exactly one source node: the loop is parallel */
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        const int x = (int)(n % nx), y = (int)(n / nx);
        if (solid2(p, x, y)) continue;
        double ft[9], gt[10], Fn[2], z2[2] = {0.0, 0.0};
        for (int d = 0; d < 2; ++d) Fn[d] = p->F[d] + (Fext ? Fext[n*2+d] : 0.0);
        node2_macro nm;
        node2_collide(p, s, tau_m, f + n*9, p->induction ? g + n*10 : NULL, p->induction ? FL + n*2 : z2, Fn,
                      ft, gt, &nm);
        if (p->induction) { FL[n*2] = nm.FL[0]; FL[n*2+1] = nm.FL[1]; }
        /* Eq. pstreaming, half-way bounce-back at solid links */
        for (int a = 0; a < 9; ++a) {
            const int xt = wrap2(x + E9[a][0], nx), yt = wrap2(y + E9[a][1], ny);
            if (solid2(p, xt, yt)) fn[n*9 + opp9(a)] = ft[a];
            else fn[((long)yt*nx + xt)*9 + a] = ft[a];
        }
        if (p->induction) {
            /* Eq. mstreaming on D2Q5, anti-bounce-back to B0 at insulating walls */
            for (int a = 0; a < 5; ++a) {
                const int xt = wrap2(x + E5[a][0], nx), yt = wrap2(y + E5[a][1], ny);
                const int sol = solid2(p, xt, yt);
                const long tn = (long)yt*nx + xt;
                for (int j = 0; j < 2; ++j) {
                    if (sol) gn[n*10 + j*5 + opp5(a)] = -gt[j*5+a] + 2.0*W5(a)*p->B0[j];
                    else gn[tn*10 + j*5 + a] = gt[j*5+a];
                }
            }
        }
    }
}

/* Time march with the residual of Sec. 5 every 10 levels, as orc_run:
   hist rows (t, r, num, den, mass, Mx, My, 0). */
long orc2_run(const orc2_params* p, double* f, double* g, double* FL, const double* Fext, double* usnap,
              long* tsnap, long t0, long nsteps, double tol, double* hist, long hist_cap, long* nhist)
{
    build2();
    double s[9];
    orc2_relaxation_rates(p, s);
    const double tau_m = p->induction ? orc2_tau_m(p) : 1.0;
    const long N = (long)p->nx*p->ny;
    double* fn = (double*)malloc(sizeof(double)*9*N);
    double* gn = p->induction ? (double*)malloc(sizeof(double)*10*N) : NULL;
    double* ut = (double*)malloc(sizeof(double)*2*N);
    double* rh = (double*)malloc(sizeof(double)*N);
    long nh = nhist ? *nhist : 0, t = t0;
    memcpy(fn, f, sizeof(double)*9*N);
    if (gn) memcpy(gn, g, sizeof(double)*10*N);
    for (; t < t0 + nsteps; ++t) {
        if (t % 10 == 0 && t != *tsnap) {
            orc2_fields(p, f, g, FL, Fext, rh, ut, NULL);
            int stop = 0;
            if (*tsnap >= 0) {
                double num = 0.0, den = 0.0, mass = 0.0, mom[2] = {0.0, 0.0};
                for (long n = 0; n < N; ++n) {
                    if (solid2(p, (int)(n % p->nx), (int)(n / p->nx))) continue;
                    for (int d = 0; d < 2; ++d) {
                        const double du = ut[n*2+d] - usnap[n*2+d];
                        num += du*du;
                        den += ut[n*2+d]*ut[n*2+d];
                        mom[d] += rh[n]*ut[n*2+d];
                    }
                    mass += rh[n];
                }
                double r = den > 0.0 ? sqrt(num/den) : (num > 0.0 ? INFINITY : 0.0);
                if (!isfinite(num) || !isfinite(den)) r = NAN;
                if (hist && nh < hist_cap) {
                    double* h = hist + nh*8;
                    h[0] = (double)t; h[1] = r; h[2] = num; h[3] = den; h[4] = mass; h[5] = mom[0]; h[6] = mom[1];
                    h[7] = 0.0;
                    ++nh;
                }
                stop = (tol > 0.0 && r <= tol) || !isfinite(r);
            }
            memcpy(usnap, ut, sizeof(double)*2*N);
            *tsnap = t;
            if (stop) break;
        }
        step2(p, s, tau_m, f, g, FL, Fext, fn, gn);
        memcpy(f, fn, sizeof(double)*9*N);
        if (gn) memcpy(g, gn, sizeof(double)*10*N);
    }
    if (nhist) *nhist = nh;
    free(fn); free(gn); free(ut); free(rh);
    return t;
}
