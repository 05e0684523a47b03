/*
 * FP64 CPU oracle for the streaming-collision lattice Boltzmann scheme with the
 * kinetic diffuse-reflection wall of Meng & Zhang, "Kinetic diffuse boundary
 * condition for high-order lattice Boltzmann model with streaming-collision
 * mechanism" (arXiv:1209.5201).
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check, and the CPU
 * baseline leg and reference arm of the benchmark are the only code allowed
 * to load it.  It
 * shares no code, header, table or helper with the CUDA library: it takes the
 * lattice tables as plain arrays from its own Python generator, and it
 * follows the paper's push / ghost-layer description step by step, with no
 * blocking, fusion or reordering beyond what the equations state.
 *
 * Units (Sec. II, Eq. (2)): velocities in sqrt(R T0), length in the channel
 * height L = 1, time in L / sqrt(R T0).  The lattice velocity is
 * c_a = r * e_a with integer e_a; a time step dt = dx / r moves population a
 * by exactly e_a cells (Sec. II, the paragraph after Eq. (5)).
 * Grid: Nx periodic columns, Ny fluid rows; row j sits at y = (j + 1/2) dx,
 * dx = 1 / Ny, so each wall lies half a cell outside the outermost fluid row
 * (Sec. III).  Bottom wall (y = 0) has normal +y, top wall (y = 1) has -y.
 *
 * Storage: f[(a * Ny + j) * Nx + x], a = velocity index, in the caller's
 * lattice order.  All sums run in ascending a, then ascending row / layer.
 *
 * Readings of the paper that this file encodes (each is also listed in the
 * design notes):
 *  - tau = sqrt(2/pi) Kn mu / p with p = rho T and mu = T^mu_exp, the local
 *    pre-collision rho and T of the cell (Sec. II; Kn as in Eq. (15)).
 *  - The wall equilibrium uses the bulk expansion order; isothermal runs use
 *    T_w = 1 (Eq. (4) with T = 1).
 *  - The layer criteria of Sec. III are applied in lattice units: incoming at
 *    layer l when e_a . n - v_n < -l, outgoing when e_a . n - v_n > l, with
 *    v_n = u_w . n / r the wall's normal velocity in cells per step (0 for
 *    the paper's tangential walls, where they are integer comparisons of
 *    e_y).  A nonzero v_n is applied on the fixed half-way geometry exactly
 *    as the criteria read; a re-emitted population whose target row is not
 *    a fluid row is counted as lost (wall statistics).
 *  - The wall acts on the transformed variable f~ as streamed (Eq. (5)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int Q;
    const int *ex;      /* Q integer x-components e_a,x */
    const int *ey;      /* Q integer y-components e_a,y */
    const double *w;    /* Q quadrature weights w_a */
    double r;           /* lattice scale: c_a = r e_a */
} orc_lattice;

typedef struct {
    int Nx, Ny;
    int eq_order;       /* 2, 3 or 4: number of Hermite orders kept in Eq. (4) */
    int thermal;        /* 0: T is fixed to 1 (isothermal) */
    double Kn;          /* Knudsen number, Eq. (15) */
    double tau;         /* > 0: constant relaxation time (units L/sqrt(R T0)) */
    double mu_exp;      /* viscosity law mu = T^mu_exp */
    double u_wall[2];   /* x-velocity of the bottom (y=0) and top (y=1) wall */
    double T_wall[2];   /* temperature of the bottom and top wall */
    double accom[2];    /* accommodation of the scattering kernel per wall:
                           R = accom R_D + (1 - accom) R_S (1: diffuse) */
    double vn[2];       /* normal wall velocity u_w . n / r per wall, in cells
                           per step (n into the gas; |vn| < 1; 0: tangential) */
} orc_params;

typedef struct {
    /* Totals over columns of the last step: incoming mass numerator of
     * Eq. (12) and the mass actually re-emitted, per wall. */
    double m_in[2];
    double m_out[2];
    long long holes_unfilled;   /* fluid slots no population reached */
    long long slots_doubled;    /* fluid slots reached twice */
    double m_lost[2];           /* re-emitted mass whose target row is no
                                   fluid row (only with a normal velocity) */
} orc_wallstats;

#define ORC_D 2  /* space dimension D of Eq. (3)-(4) */

static int orc_ghost_depth(const orc_lattice *L)
{
    /* N = largest wall-ward lattice velocity (Sec. III). */
    int n = 0;
    for (int a = 0; a < L->Q; ++a) {
        int m = abs(L->ey[a]);
        if (m > n) n = m;
    }
    return n;
}

/* Eq. (4): g_a^eq(u, T), truncated at Hermite order `order`, times rho. */
void orc_equilibrium(const orc_lattice *L, int order, double rho, double ux,
                     double uy, double T, double *feq)
{
    const double D = ORC_D;
    double u2 = ux * ux + uy * uy;
    double th = T - 1.0;
    for (int a = 0; a < L->Q; ++a) {
        double cx = L->r * L->ex[a], cy = L->r * L->ey[a];
        double cu = cx * ux + cy * uy;
        double c2 = cx * cx + cy * cy;
        double g = 1.0 + cu + 0.5 * (cu * cu - u2 + th * (c2 - D));
        if (order >= 3)
            g += cu / 6.0 * (cu * cu - 3.0 * u2 + 3.0 * th * (c2 - D - 2.0));
        if (order >= 4) {
            g += (cu * cu * cu * cu - 6.0 * cu * cu * u2 + 3.0 * u2 * u2) / 24.0;
            g += th / 4.0 * ((c2 - D - 2.0) * (cu * cu - u2) - 2.0 * cu * cu);
            g += th * th / 8.0 * (c2 * c2 - 2.0 * (D + 2.0) * c2 + D * (D + 2.0));
        }
        feq[a] = rho * L->w[a] * g;
    }
}

/* Eq. (3) applied to f~ (valid for the conserved moments, Sec. II end):
 * rho = sum f, rho u = sum c f, rho D T = sum f |c - u|^2. */
void orc_moments(const orc_lattice *L, int thermal, const double *fa,
                 long stride, double *rho, double *ux, double *uy, double *T)
{
    double s0 = 0.0, sx = 0.0, sy = 0.0;
    for (int a = 0; a < L->Q; ++a) {
        double v = fa[a * stride];
        s0 += v;
        sx += L->r * L->ex[a] * v;
        sy += L->r * L->ey[a] * v;
    }
    double u = sx / s0, v = sy / s0;
    double t = 1.0;
    if (thermal) {
        double e = 0.0;
        for (int a = 0; a < L->Q; ++a) {
            double Cx = L->r * L->ex[a] - u, Cy = L->r * L->ey[a] - v;
            e += fa[a * stride] * (Cx * Cx + Cy * Cy);
        }
        t = e / (s0 * ORC_D);
    }
    *rho = s0; *ux = u; *uy = v; *T = t;
}

/* Time step dt = dx / r with dx = 1 / Ny. */
static double orc_dt(const orc_lattice *L, const orc_params *P)
{
    return 1.0 / (L->r * P->Ny);
}

/* Local relaxation time tau = sqrt(2/pi) Kn mu / (rho T) (Sec. II, Eq. (15)),
 * or the constant one. */
static double orc_tau(const orc_params *P, double rho, double T)
{
    if (P->tau > 0.0) return P->tau;
    double mu = pow(T, P->mu_exp);
    return sqrt(2.0 / M_PI) * P->Kn * mu / (rho * T);
}

/* Relaxation factor dt / (tau + dt/2) of Eq. (5). */
static double orc_omega(const orc_lattice *L, const orc_params *P, double rho,
                        double T)
{
    double dt = orc_dt(L, P);
    return dt / (orc_tau(P, rho, T) + 0.5 * dt);
}

/* Collision half of Eq. (5), in place on every fluid cell:
 * f~* = f~ - dt/(tau + dt/2) (f~ - f^eq). */
void orc_collide(const orc_lattice *L, const orc_params *P, double *f)
{
    const long plane = (long)P->Nx * P->Ny;
    const int Q = L->Q;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < plane; ++c) {
        double feq[64];
        double rho, ux, uy, T;
        orc_moments(L, P->thermal, f + c, plane, &rho, &ux, &uy, &T);
        double om = orc_omega(L, P, rho, T);
        orc_equilibrium(L, P->eq_order, rho, ux, uy, P->thermal ? T : 1.0, feq);
        for (int a = 0; a < Q; ++a) {
            double v = f[a * plane + c];
            f[a * plane + c] = v - om * (v - feq[a]);
        }
    }
}

/* Wall distribution g_a^eq(u_w, T_w) of Eq. (11)-(12) and its normalising
 * double sum over ghost layers l = 0..N-1 and outgoing velocities
 * (e_a . n > l), written as the literal double loop. wall: 0 bottom, 1 top. */
double orc_wall_distribution(const orc_lattice *L, const orc_params *P,
                             int wall, double *gw)
{
    double Tw = P->thermal ? P->T_wall[wall] : 1.0;
    int nsgn = wall == 0 ? 1 : -1;     /* normal into the gas: +y / -y */
    /* the wall velocity: tangential u_wall, normal vn r along n */
    orc_equilibrium(L, P->eq_order, 1.0, P->u_wall[wall], nsgn * P->vn[wall] * L->r, Tw, gw);
    int N = orc_ghost_depth(L);
    double den = 0.0;
    for (int l = 0; l < N; ++l)
        for (int a = 0; a < L->Q; ++a)
            if (nsgn * L->ey[a] - P->vn[wall] > l) den += gw[a];
    return den;
}

/* One time step in the paper's order: collide (Eq. (5) right-hand side),
 * push-stream into an extended grid with N ghost rows per wall, evaluate
 * Eq. (12) per ghost column, push the re-emitted populations from the ghost
 * rows into the fluid.  f holds pre-collision f~ on entry and on exit. */
static int orc_one_step(const orc_lattice *L, const orc_params *P, double *f,
                        double *ext, unsigned char *hits, orc_wallstats *st)
{
    const int Q = L->Q, Nx = P->Nx, Ny = P->Ny;
    const int N = orc_ghost_depth(L);
    const int Ne = Ny + 2 * N;                   /* extended rows */
    const long plane = (long)Nx * Ny;
    const long eplane = (long)Nx * Ne;

    orc_collide(L, P, f);

    memset(ext, 0, sizeof(double) * eplane * Q);
    memset(hits, 0, (size_t)plane * Q);

    /* Push-stream: (x, j) -> (x + e_x mod Nx, j + e_y); rows j + e_y < 0 or
     * >= Ny are ghost rows and receive the incoming populations f^I. */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < Ny; ++j) {
        for (int a = 0; a < Q; ++a) {
            int tj = j + L->ey[a];
            for (int x = 0; x < Nx; ++x) {
                int tx = ((x + L->ex[a]) % Nx + Nx) % Nx;
                ext[a * eplane + (long)(tj + N) * Nx + tx] =
                    f[a * plane + (long)j * Nx + x];
                if (tj >= 0 && tj < Ny) hits[a * plane + (long)tj * Nx + tx] += 1;
            }
        }
    }

    double gw[2][64], den[2];
    den[0] = orc_wall_distribution(L, P, 0, gw[0]);
    den[1] = orc_wall_distribution(L, P, 1, gw[1]);
    double tot_in[2] = {0.0, 0.0}, tot_out[2] = {0.0, 0.0}, lost[2] = {0.0, 0.0};

    for (int wall = 0; wall < 2; ++wall) {
        int nsgn = wall == 0 ? 1 : -1;
        const double vn = P->vn[wall];
        for (int xw = 0; xw < Nx; ++xw) {
            /* ghost layer l sits at fluid row -1-l (bottom) or Ny+l (top) */
            double m_in = 0.0;
            for (int l = 0; l < N; ++l) {
                int grow = wall == 0 ? -1 - l : Ny + l;
                for (int a = 0; a < Q; ++a)
                    if (nsgn * L->ey[a] - vn < -l)  /* incoming at layer l */
                        m_in += ext[a * eplane + (long)(grow + N) * Nx + xw];
            }
            tot_in[wall] += m_in;
            /* Eq. (9) with R = accom R_D + (1 - accom) R_S.  R_D is Eq. (11),
             * giving Eq. (12): the same diffuse f^O on every layer the velocity
             * leaves from.  R_S (specular) sends the incoming population of
             * the mirrored velocity (e_x, -e_y) at the same ghost node and
             * layer to the outgoing velocity.  Both satisfy Eq. (10). */
            const double acc = P->accom[wall];
            double fspec[64 * 3];
            for (int l = 0; l < N; ++l) {
                int grow = wall == 0 ? -1 - l : Ny + l;
                for (int a = 0; a < Q; ++a) {
                    fspec[a * N + l] = 0.0;
                    if (!(nsgn * L->ey[a] - vn > l)) continue;
                    for (int b = 0; b < Q; ++b)
                        if (L->ex[b] == L->ex[a] && L->ey[b] == -L->ey[a])
                            fspec[a * N + l] = ext[b * eplane + (long)(grow + N) * Nx + xw];
                }
            }
            for (int l = 0; l < N; ++l) {
                int grow = wall == 0 ? -1 - l : Ny + l;
                for (int a = 0; a < Q; ++a) {
                    if (!(nsgn * L->ey[a] - vn > l)) continue;   /* outgoing */
                    double fo = acc * (m_in * gw[wall][a] / den[wall]) +
                                (1.0 - acc) * fspec[a * N + l];
                    tot_out[wall] += fo;
                    int tj = grow + L->ey[a];
                    int tx = ((xw + L->ex[a]) % Nx + Nx) % Nx;
                    if (tj < 0 || tj >= Ny) {
                        /* only with vn < 0: a population with e.n = l leaving
                         * layer l lands in a ghost row again */
                        if (vn == 0.0) return -1;
                        lost[wall] += fo;
                        continue;
                    }
                    ext[a * eplane + (long)(tj + N) * Nx + tx] = fo;
                    hits[a * plane + (long)tj * Nx + tx] += 1;
                }
            }
        }
    }

    long long unfilled = 0, doubled = 0;
    for (long i = 0; i < plane * Q; ++i) {
        if (hits[i] == 0) ++unfilled;
        if (hits[i] > 1) ++doubled;
    }
    for (int a = 0; a < Q; ++a)
        memcpy(f + a * plane, ext + a * eplane + (long)N * Nx,
               sizeof(double) * plane);

    if (st) {
        for (int k = 0; k < 2; ++k) {
            st->m_in[k] = tot_in[k];
            st->m_out[k] = tot_out[k];
            st->m_lost[k] = lost[k];
        }
        st->holes_unfilled = unfilled;
        st->slots_doubled = doubled;
    }
    return (unfilled || doubled) ? -2 : 0;
}

/* Advance f (pre-collision f~) by nsteps.  Returns 0, or a negative code if
 * the ghost-layer bookkeeping ever left a fluid slot empty or doubled. */
int orc_run(const orc_lattice *L, const orc_params *P, double *f, long nsteps,
            orc_wallstats *st)
{
    if (L->Q > 64 || P->Nx < 1 || P->Ny < 1 || orc_ghost_depth(L) > 3) return -3;
    const int N = orc_ghost_depth(L);
    const long plane = (long)P->Nx * P->Ny;
    double *ext = malloc(sizeof(double) * (long)P->Nx * (P->Ny + 2 * N) * L->Q);
    unsigned char *hits = malloc((size_t)plane * L->Q);
    if (!ext || !hits) { free(ext); free(hits); return -4; }
    int rc = 0;
    for (long n = 0; n < nsteps && rc == 0; ++n)
        rc = orc_one_step(L, P, f, ext, hits, st);
    free(ext);
    free(hits);
    return rc;
}

/* Initial state f~ = rho g^eq(u, T) per cell (Eq. (4)); NULL fields mean
 * u = 0, T = 1.  rho must be given. */
void orc_init_fields(const orc_lattice *L, const orc_params *P,
                     const double *rho, const double *ux, const double *uy,
                     const double *T, double *f)
{
    const long plane = (long)P->Nx * P->Ny;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < plane; ++c) {
        double feq[64];
        orc_equilibrium(L, P->eq_order, rho[c], ux ? ux[c] : 0.0,
                        uy ? uy[c] : 0.0, T ? T[c] : 1.0, feq);
        for (int a = 0; a < L->Q; ++a) f[a * plane + c] = feq[a];
    }
}

/* Macroscopic fields of Eq. (3) for every cell. */
void orc_macros(const orc_lattice *L, const orc_params *P, const double *f,
                double *rho, double *ux, double *uy, double *T)
{
    const long plane = (long)P->Nx * P->Ny;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < plane; ++c)
        orc_moments(L, P->thermal, f + c, plane, rho + c, ux + c, uy + c, T + c);
}

/* Eq. (3) fields with the kinetic temperature sum f |c - u|^2 / (D rho) for
 * every run, isothermal ones included (there it is a diagnostic only: the
 * collision of an isothermal run uses T = 1). */
void orc_macros_kinetic(const orc_lattice *L, const orc_params *P, const double *f,
                        double *rho, double *ux, double *uy, double *T)
{
    const long plane = (long)P->Nx * P->Ny;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < plane; ++c)
        orc_moments(L, 1, f + c, plane, rho + c, ux + c, uy + c, T + c);
}

/* Stress and heat flux of every cell from its pre-collision f~.  The
 * transformed variable of Sec. II is f~ = f + dt/(2 tau) (f - f^eq), so the
 * distribution itself is f = (f~ + dt/(2 tau) f^eq) / (1 + dt/(2 tau)); its
 * central moments give
 *   sigma_ij = sum_a (c_i - u_i)(c_j - u_j) f_a - rho T delta_ij,
 *   q_i      = 1/2 sum_a |c - u|^2 (c_i - u_i) f_a,
 * with rho, u, T the conserved moments of f~ (equal to those of f) and T = 1
 * in an isothermal run (the temperature its equilibrium and tau use).
 * Outputs are [Ny][Nx] planes; any may be NULL. */
void orc_fluxes(const orc_lattice *L, const orc_params *P, const double *f,
                double *sxx, double *sxy, double *syy, double *qx, double *qy)
{
    const long plane = (long)P->Nx * P->Ny;
    const double dt = orc_dt(L, P);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < plane; ++c) {
        double feq[64];
        double rho, ux, uy, T;
        orc_moments(L, P->thermal, f + c, plane, &rho, &ux, &uy, &T);
        if (!P->thermal) T = 1.0;
        orc_equilibrium(L, P->eq_order, rho, ux, uy, T, feq);
        double h = dt / (2.0 * orc_tau(P, rho, T));
        double pxx = 0.0, pxy = 0.0, pyy = 0.0, hx = 0.0, hy = 0.0;
        for (int a = 0; a < L->Q; ++a) {
            double fa = (f[a * plane + c] + h * feq[a]) / (1.0 + h);
            double Cx = L->r * L->ex[a] - ux, Cy = L->r * L->ey[a] - uy;
            double C2 = Cx * Cx + Cy * Cy;
            pxx += Cx * Cx * fa;
            pxy += Cx * Cy * fa;
            pyy += Cy * Cy * fa;
            hx += 0.5 * C2 * Cx * fa;
            hy += 0.5 * C2 * Cy * fa;
        }
        if (sxx) sxx[c] = pxx - rho * T;
        if (sxy) sxy[c] = pxy;
        if (syy) syy[c] = pyy - rho * T;
        if (qx) qx[c] = hx;
        if (qy) qy[c] = hy;
    }
}

/* Steady-state driver: run in chunks of check_every steps until the relative
 * change of u_x over one chunk (and, when thermal, of T - T_ref) drops to
 * tol.  Returns 0 when converged, 1 when max_steps ran out, < 0 on error. */
int orc_run_to_residual(const orc_lattice *L, const orc_params *P, double *f,
                        double tol, long max_steps, int check_every,
                        long *steps_done, double *res_out)
{
    const long plane = (long)P->Nx * P->Ny;
    double *m = malloc(sizeof(double) * plane * 6);
    if (!m) return -4;
    double *rho = m, *ux = m + plane, *uy = m + 2 * plane, *T = m + 3 * plane;
    double *ux0 = m + 4 * plane, *T0 = m + 5 * plane;
    double Tref = 0.5 * (P->T_wall[0] + P->T_wall[1]);
    orc_macros(L, P, f, rho, ux0, uy, T0);
    long n = 0;
    double res = INFINITY;
    int rc = 1;
    while (n < max_steps) {
        long k = check_every;
        if (n + k > max_steps) k = max_steps - n;
        int e = orc_run(L, P, f, k, NULL);
        if (e) { rc = e; break; }
        n += k;
        orc_macros(L, P, f, rho, ux, uy, T);
        double du = 0.0, nu = 0.0, dT = 0.0, nT = 0.0;
        for (long c = 0; c < plane; ++c) {
            du += (ux[c] - ux0[c]) * (ux[c] - ux0[c]);
            nu += ux[c] * ux[c];
            dT += (T[c] - T0[c]) * (T[c] - T0[c]);
            nT += (T[c] - Tref) * (T[c] - Tref);
        }
        res = sqrt(du) / fmax(sqrt(nu), 1e-30);
        if (P->thermal) {
            double rt = sqrt(dT) / fmax(sqrt(nT), 1e-30);
            if (rt > res) res = rt;
        }
        memcpy(ux0, ux, sizeof(double) * plane);
        memcpy(T0, T, sizeof(double) * plane);
        if (!(res == res)) { rc = -5; break; }
        if (res <= tol) { rc = 0; break; }
    }
    free(m);
    *steps_done = n;
    *res_out = res;
    return rc;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops from now on (timing on one core or all). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
