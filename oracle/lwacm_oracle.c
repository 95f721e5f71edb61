/*
 * FP64 CPU oracle for the Link-wise Artificial Compressibility Method (LW-ACM).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call this file:
 * only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * load it. It shares no code, header or table with the CUDA library.
 *
 * What it computes, and where the paper defines it (Asinari et al., "Link-wise
 * Artificial Compressibility Method"):
 *   - lattices D2Q9 / D3Q19 and the second-order equilibrium f_i^(e)
 *     (Appendix "Equilibrium distribution functions", Eq. d2q9_equilibrium_compact,
 *     Eq. weight_factors, Eq. weight_factors_3d);
 *   - the odd part f_i^(e,o) = (f^(e)(rho,u) - f^(e)(rho,-u))/2 (Eq. feqo);
 *   - the update, written in the populations form of Eq. ACM2.0:
 *       f_i(x,t+1) = f_i^(e)(x-c_i,t) + 2(omega-1)/omega [f_i^(e,o)(x,t) - f_i^(e,o)(x-c_i,t)]
 *     followed by rho = sum_i f_i, rho u = sum_i c_i f_i (Section 2.1);
 *   - omega from nu by Eq. viscosity2, nu = (1/omega - 1/2)/3;
 *   - half-way link-wise walls, Eq. ACM2.0cccbb2, with the moving-wall term of
 *     Eq. ACM2.0ccccbb (Section 2.6, rules of the 2D cavity in Section 2.6.1);
 *   - a passive scalar advected and diffused by Eq. ACM2.0t (lwo_step_scalar);
 *   - a separate relaxation frequency omega_p for the pressure update (Section
 *     2.2, item 3), periodic domains (lwo_step_nu_p);
 *   - the semi-implicit pressure update of Eq. FDcompact_si (Section 2.2, item 2),
 *     periodic domains (lwo_step_semi_implicit);
 *   - the bulk-viscosity variant of Appendix "Computing derivatives locally"
 *     (Eq. quasi-equilibrium2 with the quasi-equilibrium of Eq. quasi-equilibrium
 *     and the product form of Eq. d2q9_equilibrium_gen), D2Q9, periodic
 *     (lwo_step_bulk);
 *   - external forcing, Eq. force, with a constant acceleration or a per-node
 *     field g(x) (lwo_step_force_field; a time-dependent g is applied by one call
 *     per step);
 *   - an equilibrium-initialised BGK lattice Boltzmann comparator (the LKS limit
 *     omega = 1 named in Section 2.2);
 *   - the D2Q9 finite-difference formulas Eqs. FDjx, FDjy, FDpressure (Appendix C);
 *   - the reverse-mode derivative (adjoint) of the populations-form step, by the
 *     chain rule applied to the definitions above, and a gradient driver for the
 *     loss 0.5 sum |u(T) - u_target|^2.
 *
 * Arithmetic is FP64, scalar loops, no blocking or fusion. Fields are stored
 * [nz][ny][nx], x fastest; d = rho - 1.
 *
 * Parity status: every function here is pinned by the CPU test-suite (exact
 * identities, closed forms, brute-force derivatives); see the test files.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define LWO_MAXQ 19

enum { LWO_PERIODIC = 0, LWO_CAVITY = 1, LWO_CHANNEL = 2 };

typedef struct {
    int Q, D;
    int c[LWO_MAXQ][3];
    double w[LWO_MAXQ];
    int bb[LWO_MAXQ];
} lwo_lattice;

/* D2Q9, index order of the explicit equilibria in Appendix "Equilibrium
 * distribution functions": rest, +x, +y, -x, -y, (1,1), (-1,1), (-1,-1), (1,-1);
 * weights 4/9, 1/9, 1/36 (Eq. weight_factors). */
static void make_d2q9(lwo_lattice *L) {
    static const int c[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    L->Q = 9;
    L->D = 2;
    for (int i = 0; i < 9; ++i) {
        L->c[i][0] = c[i][0];
        L->c[i][1] = c[i][1];
        L->c[i][2] = 0;
        L->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
}

/* D3Q19: rest; the six axis links; the twelve face diagonals (Appendix
 * "Equilibrium distribution functions", weights 1/3, 1/18, 1/36 by
 * Eq. weight_factors_3d). The paper gives no index order; this one keeps each
 * link next to its opposite. */
static void make_d3q19(lwo_lattice *L) {
    static const int c[19][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    L->Q = 19;
    L->D = 3;
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) L->c[i][a] = c[i][a];
        L->w[i] = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
}

static int make_lattice(int Q, lwo_lattice *L) {
    if (Q == 9)
        make_d2q9(L);
    else if (Q == 19)
        make_d3q19(L);
    else
        return -1;
    /* bounce-back operator BB(i): the link with c_BB(i) = -c_i (Section 2.6) */
    for (int i = 0; i < L->Q; ++i) {
        L->bb[i] = -1;
        for (int j = 0; j < L->Q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] &&
                L->c[j][2] == -L->c[i][2])
                L->bb[i] = j;
    }
    return 0;
}

/* Eq. d2q9_equilibrium_compact: f_i^(e) = w_i rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2];
 * "formally identical" for D3Q19. */
static double feq(const lwo_lattice *L, int i, double rho, const double u[3]) {
    const double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return L->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* Eq. feqo: the odd part, evaluated from its definition. */
static double feqo(const lwo_lattice *L, int i, double rho, const double u[3]) {
    const double mu[3] = {-u[0], -u[1], -u[2]};
    return 0.5 * (feq(L, i, rho, u) - feq(L, i, rho, mu));
}

/* d f^(e) / d rho and d f^(e) / d u_a (derivatives of the polynomial above). */
static double feq_drho(const lwo_lattice *L, int i, const double u[3]) {
    const double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return L->w[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}
static double feq_du(const lwo_lattice *L, int i, double rho, const double u[3], int a) {
    const double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
    return L->w[i] * rho * (3.0 * L->c[i][a] + 9.0 * cu * L->c[i][a] - 3.0 * u[a]);
}
/* chain rule through Eq. feqo: d/du of f^(e)(rho,-u) is -(df^(e)/du)(rho,-u) */
static double feqo_drho(const lwo_lattice *L, int i, const double u[3]) {
    const double mu[3] = {-u[0], -u[1], -u[2]};
    return 0.5 * (feq_drho(L, i, u) - feq_drho(L, i, mu));
}
static double feqo_du(const lwo_lattice *L, int i, double rho, const double u[3], int a) {
    const double mu[3] = {-u[0], -u[1], -u[2]};
    return 0.5 * (feq_du(L, i, rho, u, a) + feq_du(L, i, rho, mu, a));
}

typedef struct {
    int n[3];
    int walled[3]; /* 1 = half-way walls on both ends of this axis */
    int lid_axis;  /* the wall at the top of this axis moves with the lid velocity */
} lwo_geom;

static int make_geom(const lwo_lattice *L, int nx, int ny, int nz, int bc, lwo_geom *G) {
    if (nx < 1 || ny < 1 || nz < 1) return -2;
    if (L->D == 2 && nz != 1) return -2;
    G->n[0] = nx;
    G->n[1] = ny;
    G->n[2] = nz;
    G->walled[0] = G->walled[1] = G->walled[2] = 0;
    G->lid_axis = L->D - 1;
    if (bc == LWO_CAVITY) {
        for (int a = 0; a < L->D; ++a) G->walled[a] = 1;
    } else if (bc == LWO_CHANNEL) {
        G->walled[1] = 1;
        G->lid_axis = 1;
    } else if (bc != LWO_PERIODIC) {
        return -3;
    }
    return 0;
}

/* Source node s = x - c_i. Returns its linear index, or -1 when it falls outside
 * the grid across a wall; *above_lid is set when that outside point lies beyond
 * the top wall of the lid axis. Periodic axes wrap. */
static long source_of(const lwo_geom *G, const int x[3], const int c[3], int *above_lid) {
    int s[3];
    *above_lid = 0;
    int outside = 0;
    for (int a = 0; a < 3; ++a) {
        s[a] = x[a] - c[a];
        if (s[a] < 0 || s[a] >= G->n[a]) {
            if (G->walled[a]) {
                outside = 1;
                if (a == G->lid_axis && s[a] >= G->n[a]) *above_lid = 1;
            } else {
                s[a] = ((s[a] % G->n[a]) + G->n[a]) % G->n[a];
            }
        }
    }
    if (outside) return -1;
    return ((long)s[2] * G->n[1] + s[1]) * G->n[0] + s[0];
}

static void load_u(const double *ux, const double *uy, const double *uz, long k, double u[3]) {
    u[0] = ux[k];
    u[1] = uy[k];
    u[2] = uz ? uz[k] : 0.0;
}

/* One node of Eq. ACM2.0 (with walls and forcing): writes rho(x,t+1), u(x,t+1).
 * omega_p: the relaxation frequency of the pressure (density) update (Section 2.2,
 * item 3: Eq. FDcompact c with omega_p); the density sums populations built with
 * a_p = 2(omega_p-1)/omega_p, the momentum those built with a (periodic links). */
static void node_update(const lwo_lattice *L, const lwo_geom *G, double omega, double omega_p, double rho0,
                        const double lid[3], const double force[3], int has_force, const int x[3],
                        const double *d, const double *ux, const double *uy, const double *uz,
                        double *rho_new, double u_new[3]) {
    const long k = ((long)x[2] * G->n[1] + x[1]) * G->n[0] + x[0];
    const double a = 2.0 * (omega - 1.0) / omega;  /* Eq. ACM2.0 */
    const double ap = 2.0 * (omega_p - 1.0) / omega_p;
    const double bw = 2.0 / omega - 1.0;           /* Eq. ACM2.0ccccbb */
    const double zero[3] = {0.0, 0.0, 0.0};
    double ux_[3];
    load_u(ux, uy, uz, k, ux_);
    const double rx = 1.0 + d[k];
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->Q; ++i) {
        int above;
        const long s = source_of(G, x, L->c[i], &above);
        double f, fp;
        if (s >= 0) {
            double us[3];
            load_u(ux, uy, uz, s, us);
            const double rs = 1.0 + d[s];
            f = feq(L, i, rs, us) + a * (feqo(L, i, rx, ux_) - feqo(L, i, rs, us));
            fp = feq(L, i, rs, us) + ap * (feqo(L, i, rx, ux_) - feqo(L, i, rs, us));
        } else {
            /* link i arrives from outside: Eq. ACM2.0cccbb2 with BB(i) pointing at
             * the wall, plus the moving-wall correction of Eq. ACM2.0ccccbb */
            const int j = L->bb[i];
            const double *uw = above ? lid : zero;
            f = feq(L, j, rx, ux_) + (2.0 - 2.0 / omega) * 2.0 * feqo(L, i, rx, ux_) +
                bw * 2.0 * feqo(L, i, rho0, uw);
            fp = f;
        }
        if (has_force) {
            f += feqo(L, i, rx, force); /* Eq. force */
            fp += feqo(L, i, rx, force);
        }
        rho += fp;
        for (int b = 0; b < 3; ++b) m[b] += L->c[i][b] * f;
    }
    *rho_new = rho;
    for (int b = 0; b < 3; ++b) u_new[b] = m[b] / rho;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int lwo_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double omega_of_nu(double nu) { return 2.0 / (6.0 * nu + 1.0); } /* Eq. viscosity2 */

/* Advance (d,ux,uy[,uz]) in place by nsteps of Eq. ACM2.0, with the external
 * acceleration g of Eq. force either one constant vector (force, or NULL) or, when
 * gx is not NULL, a per-node field (gx, gy[, gz]) held fixed over the nsteps. */
static int run_steps(int Q, int nx, int ny, int nz, double nu, double nu_p, int bc, double rho0,
                     const double *lid, const double *force, const double *gx, const double *gy,
                     const double *gz, long nsteps, double *d, double *ux, double *uy, double *uz,
                     int nthreads) {
    lwo_lattice L;
    lwo_geom G;
    if (make_lattice(Q, &L)) return -1;
    if (make_geom(&L, nx, ny, nz, bc, &G)) return -2;
    if (!(nu > 0.0)) return -4;
    if (Q == 19 && !uz) return -5;
    if (gx && !gy) return -3;
    if (!(nu_p > 0.0)) return -4;
    if (nu_p != nu && bc != LWO_PERIODIC) return -7; /* omega_p only on periodic domains */
    set_threads(nthreads);
    const double omega = omega_of_nu(nu), omega_p = omega_of_nu(nu_p);
    const double zero[3] = {0.0, 0.0, 0.0};
    const double *lid_ = lid ? lid : zero;
    const double *frc = force ? force : zero;
    const int has_force =
        gx != NULL || (force && (force[0] != 0.0 || force[1] != 0.0 || force[2] != 0.0));
    const long N = (long)nx * ny * nz;
    const int nf = (Q == 19) ? 4 : 3;
    double *buf = (double *)malloc(sizeof(double) * N * nf);
    if (!buf) return -6;
    double *src[4] = {d, ux, uy, uz};
    double *dst[4] = {buf, buf + N, buf + 2 * N, (nf == 4) ? buf + 3 * N : NULL};
    for (long t = 0; t < nsteps; ++t) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int xx = 0; xx < nx; ++xx) {
                    const int x[3] = {xx, y, z};
                    const long k = ((long)z * ny + y) * nx + xx;
                    double r, u[3], gk[3];
                    const double *g = frc;
                    if (gx) {
                        gk[0] = gx[k];
                        gk[1] = gy[k];
                        gk[2] = gz ? gz[k] : 0.0;
                        g = gk;
                    }
                    node_update(&L, &G, omega, omega_p, rho0, lid_, g, has_force, x, src[0], src[1],
                                src[2], src[3], &r, u);
                    dst[0][k] = r - 1.0;
                    dst[1][k] = u[0];
                    dst[2][k] = u[1];
                    if (dst[3]) dst[3][k] = u[2];
                }
        for (int f = 0; f < 4; ++f) {
            double *tmp = src[f];
            src[f] = dst[f];
            dst[f] = tmp;
        }
    }
    if (src[0] != d) {
        double *orig[4] = {d, ux, uy, uz};
        for (int f = 0; f < nf; ++f) memcpy(orig[f], src[f], sizeof(double) * N);
    }
    free(buf);
    return 0;
}

/* Advance (d,ux,uy[,uz]) in place by nsteps of Eq. ACM2.0. rho0 enters only the
 * moving-wall term. lid / force may be NULL (zero). Returns 0 or a negative code. */
int lwo_step(int Q, int nx, int ny, int nz, double nu, int bc, double rho0, const double *lid,
             const double *force, long nsteps, double *d, double *ux, double *uy, double *uz,
             int nthreads) {
    return run_steps(Q, nx, ny, nz, nu, nu, bc, rho0, lid, force, NULL, NULL, NULL, nsteps, d, ux, uy,
                     uz, nthreads);
}

/* As lwo_step, with a per-node acceleration field g(x) = (gx, gy[, gz]) (Eq. force
 * written for a space-dependent g), held fixed over the nsteps; a time-dependent
 * g(x,t) is applied by one call per step with g evaluated at time t. gz may be
 * NULL (zero). */
int lwo_step_force_field(int Q, int nx, int ny, int nz, double nu, int bc, double rho0,
                         const double *lid, const double *gx, const double *gy, const double *gz,
                         long nsteps, double *d, double *ux, double *uy, double *uz, int nthreads) {
    if (!gx || !gy) return -3;
    return run_steps(Q, nx, ny, nz, nu, nu, bc, rho0, lid, NULL, gx, gy, gz, nsteps, d, ux, uy, uz,
                     nthreads);
}

/* As lwo_step / lwo_step_force_field on a periodic domain, with a separate
 * viscosity nu_p for the pressure (density) update (omega_p of Section 2.2, item 3).
 * force (constant) or gx, gy[, gz] (per node) may be NULL. */
int lwo_step_nu_p(int Q, int nx, int ny, int nz, double nu, double nu_p, const double *force,
                  const double *gx, const double *gy, const double *gz, long nsteps, double *d, double *ux,
                  double *uy, double *uz, int nthreads) {
    return run_steps(Q, nx, ny, nz, nu, nu_p, LWO_PERIODIC, 1.0, NULL, force, gx, gy, gz, nsteps, d, ux, uy, uz,
                     nthreads);
}

/* Semi-implicit pressure update (Section 2.2, item 2, Eq. FDcompact_si) on a
 * periodic domain: the density (pressure) is updated with the already updated
 * velocity, p+ = f_p(u+, p). Reading: f_u, f_v of Eq. FDcompact a, b are functions
 * of the state at t only, so u+ is the velocity of the explicit step (its momentum
 * over its explicit density); the density is then the density of Eq. ACM2.0 summed
 * again, every population built from the old density and the new velocity:
 *   rho+(x) = sum_i f_i^(e)(rho(x-c_i), u+(x-c_i))
 *             + a [f_i^(e,o)(rho(x), u+(x)) - f_i^(e,o)(rho(x-c_i), u+(x-c_i))].
 * The final state is (rho+, u+). A per-node acceleration (gx, gy[, gz], or NULL)
 * enters the momentum as in Eq. force; it leaves every density untouched, since
 * the odd parts sum to zero. */
int lwo_step_semi_implicit(int Q, int nx, int ny, int nz, double nu, const double *gx, const double *gy,
                           const double *gz, long nsteps, double *d, double *ux, double *uy, double *uz,
                           int nthreads) {
    lwo_lattice L;
    lwo_geom G;
    if (make_lattice(Q, &L)) return -1;
    if (make_geom(&L, nx, ny, nz, LWO_PERIODIC, &G)) return -2;
    if (!(nu > 0.0)) return -4;
    if (Q == 19 && !uz) return -5;
    if (gx && !gy) return -3;
    set_threads(nthreads);
    const double omega = omega_of_nu(nu);
    const double zero[3] = {0.0, 0.0, 0.0};
    const long N = (long)nx * ny * nz;
    const int nf = (Q == 19) ? 4 : 3;
    double *buf = (double *)malloc(sizeof(double) * N * nf);
    if (!buf) return -6;
    double *un[3] = {buf + N, buf + 2 * N, (nf == 4) ? buf + 3 * N : NULL};
    for (long t = 0; t < nsteps; ++t) {
        /* the explicit step: (rho+ explicit, u+) */
#pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int xx = 0; xx < nx; ++xx) {
                    const int x[3] = {xx, y, z};
                    const long k = ((long)z * ny + y) * nx + xx;
                    double r, u[3], gk[3] = {0.0, 0.0, 0.0};
                    if (gx) {
                        gk[0] = gx[k];
                        gk[1] = gy[k];
                        gk[2] = gz ? gz[k] : 0.0;
                    }
                    node_update(&L, &G, omega, omega, 1.0, zero, gk, gx != NULL, x, d, ux, uy, uz, &r, u);
                    buf[k] = r - 1.0;
                    un[0][k] = u[0];
                    un[1][k] = u[1];
                    if (un[2]) un[2][k] = u[2];
                }
        /* the density again, from the old density and the new velocity */
#pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int xx = 0; xx < nx; ++xx) {
                    const int x[3] = {xx, y, z};
                    const long k = ((long)z * ny + y) * nx + xx;
                    double r, u[3];
                    node_update(&L, &G, omega, omega, 1.0, zero, zero, 0, x, d, un[0], un[1], un[2], &r, u);
                    buf[k] = r - 1.0; /* over the explicit density, which this pass does not read */
                }
        memcpy(d, buf, sizeof(double) * N);
        memcpy(ux, un[0], sizeof(double) * N);
        memcpy(uy, un[1], sizeof(double) * N);
        if (uz) memcpy(uz, un[2], sizeof(double) * N);
    }
    free(buf);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Passive scalar (Appendix "Asymptotic analysis for energy equation", Eq. ACM2.0t):
 *   g_i(x,t+1) = g_i^(e)(x-c_i,t) + 2(omega_t-1)/omega_t [g_i^(e,e)(x,t) - g_i^(e,e)(x-c_i,t)]
 * with T = sum_i g_i advected by the flow velocity u(x,t) and diffused with
 * alpha = (1/omega_t - 1/2)/3 (Eq. diffusivity2). The equilibrium satisfies the
 * stated moments sum g^(e) = T, sum c g^(e) = T u, sum c c g^(e) = u u + T/3 I:
 *   g_i^(e)(T,u) = w_i [T (1 + 3 c_i.u) + 9/2 (c_i.u)^2 - 3/2 |u|^2],
 * and g^(e,e) is its even part in u (Eq. feqe).
 * ------------------------------------------------------------------------- */
static double geq(const lwo_lattice *L, int i, double T, const double u[3]) {
    const double e = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
    const double q = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return L->w[i] * (T * (1.0 + 3.0 * e) + 4.5 * e * e - 1.5 * q);
}
static double geqe(const lwo_lattice *L, int i, double T, const double u[3]) {
    const double mu[3] = {-u[0], -u[1], -u[2]};
    return 0.5 * (geq(L, i, T, u) + geq(L, i, T, mu)); /* Eq. feqe */
}

/* Advance (d, u) by Eq. ACM2.0 and the scalar T by Eq. ACM2.0t (with u at the
 * time level t of each step), nsteps times, on a periodic domain; alpha > 0. */
int lwo_step_scalar(int Q, int nx, int ny, int nz, double nu, double alpha, long nsteps, double *d,
                    double *ux, double *uy, double *uz, double *T, int nthreads) {
    lwo_lattice L;
    lwo_geom G;
    if (make_lattice(Q, &L)) return -1;
    if (make_geom(&L, nx, ny, nz, LWO_PERIODIC, &G)) return -2;
    if (!(alpha > 0.0) || !T) return -4;
    const long N = (long)nx * ny * nz;
    const double omega_t = omega_of_nu(alpha); /* same relation as nu(omega) */
    const double at = 2.0 * (omega_t - 1.0) / omega_t;
    double *Tn = (double *)malloc(sizeof(double) * N);
    if (!Tn) return -6;
    set_threads(nthreads);
    for (long t = 0; t < nsteps; ++t) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int xx = 0; xx < nx; ++xx) {
                    const int x[3] = {xx, y, z};
                    const long k = ((long)z * ny + y) * nx + xx;
                    double u[3];
                    load_u(ux, uy, uz, k, u);
                    double acc = 0.0;
                    for (int i = 0; i < L.Q; ++i) {
                        int above;
                        const long s = source_of(&G, x, L.c[i], &above);
                        double us[3];
                        load_u(ux, uy, uz, s, us);
                        acc += geq(&L, i, T[s], us) + at * (geqe(&L, i, T[k], u) - geqe(&L, i, T[s], us));
                    }
                    Tn[k] = acc;
                }
        /* the flow moves on with the same step */
        const int rc = lwo_step(Q, nx, ny, nz, nu, LWO_PERIODIC, 1.0, NULL, NULL, 1, d, ux, uy, uz, nthreads);
        if (rc) {
            free(Tn);
            return rc;
        }
        memcpy(T, Tn, sizeof(double) * N);
    }
    free(Tn);
    return 0;
}

/* -------------------------------------------------------------------------
 * Bulk viscosity (Appendix "Computing derivatives locally"), D2Q9 only.
 * Eq. d2q9_equilibrium_gen: f^(g)_i(Pxx, Pyy) = rho phi_x(c_ix) phi_y(c_iy) with
 * phi_x(0) = 1 - Pxx, phi_x(+-1) = (Pxx +- u)/2 and likewise for y (the listed
 * rows written as one product, independent of the link order).
 * Eq. quasi-equilibrium: f^(qe)(rho, u, Tr) = f^(g)((Tr + u^2 - v^2)/2, (Tr - u^2 + v^2)/2).
 * Eq. quasi-equilibrium2 replaces f^(e) in Eq. ACM2.0 by the quasi-equilibrium at
 * Tr* = Tr^(e) + gamma (Tr^(+) - Tr^(e)), Tr^(e) = 2/3 + |u|^2, Tr^(+) the trace of
 * sum_i c_i c_i f_i of the updated populations over rho. Reading (the printed
 * f^(g) equals f^(e) only up to third-order terms): the increment is added to
 * f^(e),
 *   f^(e*)_i = f^(e)_i + f^(qe)_i(rho, u, Tr*) - f^(qe)_i(rho, u, Tr^(e)),
 * which has the second moment of Eq. second-quasi-equilibrium2 exactly and is
 * f^(e) itself when gamma = 0 or Tr^(+) = Tr^(e). The odd part is taken from its
 * definition, (f(rho, u) - f(rho, -u))/2, as for f^(e).
 * ------------------------------------------------------------------------- */
static double fg(int cx, int cy, double rho, double u, double v, double pxx, double pyy) {
    const double px = cx == 0 ? 1.0 - pxx : 0.5 * (pxx + cx * u);
    const double py = cy == 0 ? 1.0 - pyy : 0.5 * (pyy + cy * v);
    return rho * px * py;
}
static double fqe(int cx, int cy, double rho, double u, double v, double tr) {
    return fg(cx, cy, rho, u, v, 0.5 * (tr + u * u - v * v), 0.5 * (tr - u * u + v * v));
}
static double feq_star(const lwo_lattice *L, int i, double rho, const double u[3], double tr_plus,
                       double gamma) {
    const double tre = 2.0 / 3.0 + u[0] * u[0] + u[1] * u[1];
    const double trs = tre + gamma * (tr_plus - tre);
    const int cx = L->c[i][0], cy = L->c[i][1];
    return feq(L, i, rho, u) + fqe(cx, cy, rho, u[0], u[1], trs) - fqe(cx, cy, rho, u[0], u[1], tre);
}
static double feq_star_o(const lwo_lattice *L, int i, double rho, const double u[3], double tr_plus,
                         double gamma) {
    const double mu[3] = {-u[0], -u[1], -u[2]};
    return 0.5 * (feq_star(L, i, rho, u, tr_plus, gamma) - feq_star(L, i, rho, mu, tr_plus, gamma));
}

/* f^(qe)(rho, u, Tr) of one node (Q = 9 values, Eq. quasi-equilibrium) */
int lwo_fqe(double rho, const double *u, double tr, double *f) {
    lwo_lattice L;
    if (make_lattice(9, &L)) return -1;
    for (int i = 0; i < 9; ++i) f[i] = fqe(L.c[i][0], L.c[i][1], rho, u[0], u[1], tr);
    return 0;
}

/* f^(e*) of one node (Q = 9 values), for the tests of Eq. second-quasi-equilibrium2 */
int lwo_feq_star(double rho, const double *u, double tr_plus, double gamma, double *f) {
    lwo_lattice L;
    if (make_lattice(9, &L)) return -1;
    const double uu[3] = {u[0], u[1], 0.0};
    for (int i = 0; i < 9; ++i) f[i] = feq_star(&L, i, rho, uu, tr_plus, gamma);
    return 0;
}

/* Advance (d, u, Tr) of a periodic D2Q9 domain by Eq. ACM2.0 with f^(e*) in place
 * of f^(e), nsteps times. Tr holds Tr^(+) of the last update (the caller starts it
 * at Tr^(e) = 2/3 + |u|^2, which makes the first step the standard one). nu_p > 0:
 * with omega_p as well (Section 2.2 item 3; both together are the runs of Fig.
 * minion2): the density sums populations built with a_p, the momentum and the
 * trace those built with a; u is over the new density, Tr^(+) over the zeroth
 * moment of the populations it is the trace of (the updated distribution, built
 * with a), which is the new density when nu_p = nu. */
int lwo_step_bulk(int nx, int ny, double nu, double nu_p, double gamma, long nsteps, double *d, double *ux,
                  double *uy, double *tr, int nthreads) {
    lwo_lattice L;
    lwo_geom G;
    if (make_lattice(9, &L)) return -1;
    if (make_geom(&L, nx, ny, 1, LWO_PERIODIC, &G)) return -2;
    if (!(nu > 0.0) || nu > 1.0 / 6.0) return -3;
    if (!tr) return -4;
    const long N = (long)nx * ny;
    if (nu_p < 0.0 || nu_p > 1.0 / 6.0) return -3;
    const double omega = omega_of_nu(nu);
    const double a = 2.0 * (omega - 1.0) / omega;
    const double omega_p = nu_p > 0.0 ? omega_of_nu(nu_p) : omega;
    const double ap = 2.0 * (omega_p - 1.0) / omega_p;
    double *buf = (double *)malloc(sizeof(double) * 4 * N);
    if (!buf) return -6;
    double *dn = buf, *un = buf + N, *vn = buf + 2 * N, *tn = buf + 3 * N;
    set_threads(nthreads);
    for (long t = 0; t < nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int xx = 0; xx < nx; ++xx) {
                const int x[3] = {xx, y, 0};
                const long k = (long)y * nx + xx;
                const double rk = 1.0 + d[k];
                const double uk[3] = {ux[k], uy[k], 0.0};
                double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0, m0a = 0.0;
                for (int i = 0; i < 9; ++i) {
                    int above;
                    const long s = source_of(&G, x, L.c[i], &above);
                    const double rs = 1.0 + d[s];
                    const double us[3] = {ux[s], uy[s], 0.0};
                    const double fe = feq_star(&L, i, rs, us, tr[s], gamma);
                    const double fo = feq_star_o(&L, i, rk, uk, tr[k], gamma) - feq_star_o(&L, i, rs, us, tr[s], gamma);
                    const double fi = fe + a * fo;
                    m0 += fe + ap * fo;
                    m0a += fi;
                    m1 += L.c[i][0] * fi;
                    m2 += L.c[i][1] * fi;
                    m3 += (L.c[i][0] * L.c[i][0] + L.c[i][1] * L.c[i][1]) * fi;
                }
                dn[k] = m0 - 1.0;
                un[k] = m1 / m0;
                vn[k] = m2 / m0;
                tn[k] = m3 / m0a;
            }
        memcpy(d, dn, sizeof(double) * N);
        memcpy(ux, un, sizeof(double) * N);
        memcpy(uy, vn, sizeof(double) * N);
        memcpy(tr, tn, sizeof(double) * N);
    }
    free(buf);
    return 0;
}

int lwo_lattice_tables(int Q, int *c, double *w, int *bb) {
    lwo_lattice L;
    if (make_lattice(Q, &L)) return -1;
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
        w[i] = L.w[i];
        bb[i] = L.bb[i];
    }
    return 0;
}

/* f^(e) and f^(e,o) for all links at one state (for pin tests). */
int lwo_equilibria(int Q, double rho, const double *u, double *fe, double *feo) {
    lwo_lattice L;
    if (make_lattice(Q, &L)) return -1;
    for (int i = 0; i < Q; ++i) {
        fe[i] = feq(&L, i, rho, u);
        feo[i] = feqo(&L, i, rho, u);
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * BGK lattice Boltzmann comparator: collide f' = f - omega (f - f^(e)), then
 * stream f_i(x + c_i) = f'_i(x); half-way bounce-back with the moving-wall term
 * 2 f^(e,o)_i(rho0, u_w) for links that would leave the grid. Populations are
 * stored [i][node]. Used to pin the omega = 1 identity (Section 2.2).
 * ------------------------------------------------------------------------- */
int lwo_bgk_init(int Q, int nx, int ny, int nz, const double *d, const double *ux,
                 const double *uy, const double *uz, double *f) {
    lwo_lattice L;
    if (make_lattice(Q, &L)) return -1;
    const long N = (long)nx * ny * nz;
    for (long k = 0; k < N; ++k) {
        double u[3];
        load_u(ux, uy, uz, k, u);
        for (int i = 0; i < Q; ++i) f[i * N + k] = feq(&L, i, 1.0 + d[k], u);
    }
    return 0;
}

int lwo_bgk_step(int Q, int nx, int ny, int nz, double omega, int bc, double rho0,
                 const double *lid, long nsteps, double *f, int nthreads) {
    lwo_lattice L;
    lwo_geom G;
    if (make_lattice(Q, &L)) return -1;
    if (make_geom(&L, nx, ny, nz, bc, &G)) return -2;
    set_threads(nthreads);
    const double zero[3] = {0.0, 0.0, 0.0};
    const double *lid_ = lid ? lid : zero;
    const long N = (long)nx * ny * nz;
    double *post = (double *)malloc(sizeof(double) * N * Q);
    if (!post) return -6;
    for (long t = 0; t < nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (long k = 0; k < N; ++k) {
            double rho = 0.0, m[3] = {0.0, 0.0, 0.0}, u[3];
            for (int i = 0; i < Q; ++i) {
                rho += f[i * N + k];
                for (int b = 0; b < 3; ++b) m[b] += L.c[i][b] * f[i * N + k];
            }
            for (int b = 0; b < 3; ++b) u[b] = m[b] / rho;
            for (int i = 0; i < Q; ++i)
                post[i * N + k] = f[i * N + k] - omega * (f[i * N + k] - feq(&L, i, rho, u));
        }
#pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int xx = 0; xx < nx; ++xx) {
                    const int x[3] = {xx, y, z};
                    const long k = ((long)z * ny + y) * nx + xx;
                    for (int i = 0; i < Q; ++i) {
                        int above;
                        const long s = source_of(&G, x, L.c[i], &above);
                        if (s >= 0) {
                            f[i * N + k] = post[i * N + s];
                        } else {
                            const int j = L.bb[i];
                            f[i * N + k] = post[j * N + k] + 2.0 * feqo(&L, i, rho0, above ? lid_ : zero);
                        }
                    }
                }
    }
    free(post);
    return 0;
}

int lwo_bgk_moments(int Q, int nx, int ny, int nz, const double *f, double *d, double *ux,
                    double *uy, double *uz) {
    lwo_lattice L;
    if (make_lattice(Q, &L)) return -1;
    const long N = (long)nx * ny * nz;
    for (long k = 0; k < N; ++k) {
        double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            rho += f[i * N + k];
            for (int b = 0; b < 3; ++b) m[b] += L.c[i][b] * f[i * N + k];
        }
        d[k] = rho - 1.0;
        ux[k] = m[0] / rho;
        uy[k] = m[1] / rho;
        if (uz) uz[k] = m[2] / rho;
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Appendix C: the D2Q9 finite-difference formulas Eq. FDpressure, Eq. FDjx,
 * Eq. FDjy on a periodic grid. They are homogeneous of degree one in the
 * density symbol, which is rho here (the left-hand side p+ u+ uses the same
 * symbol). Eq. FDjy is read with a '+' in front of its 2/3(1/omega - 1)[...]
 * term, as in Eq. FDjx; the printed line lacks the operator.
 * ------------------------------------------------------------------------- */
int lwo_fd_step_d2q9(int nx, int ny, double nu, long nsteps, double *d, double *u, double *v) {
    const double om = omega_of_nu(nu);
    const double k23 = 2.0 / 3.0 * (1.0 / om - 1.0);
    const long N = (long)nx * ny;
    double *buf = (double *)malloc(sizeof(double) * 3 * N);
    if (!buf) return -6;
    double *D = d, *U = u, *V = v;
    double *Dn = buf, *Un = buf + N, *Vn = buf + 2 * N;
#define IX(i, j) ((long)((((j) % ny) + ny) % ny) * nx + ((((i) % nx) + nx) % nx))
    for (long t = 0; t < nsteps; ++t) {
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long P = IX(i, j), E = IX(i + 1, j), W = IX(i - 1, j), Nn = IX(i, j + 1),
                           S = IX(i, j - 1), NE = IX(i + 1, j + 1), NW = IX(i - 1, j + 1),
                           SE = IX(i + 1, j - 1), SW = IX(i - 1, j - 1);
                const double pP = 1.0 + D[P], pE = 1.0 + D[E], pW = 1.0 + D[W], pN = 1.0 + D[Nn],
                             pS = 1.0 + D[S], pNE = 1.0 + D[NE], pNW = 1.0 + D[NW],
                             pSE = 1.0 + D[SE], pSW = 1.0 + D[SW];
                const double uP = U[P], uE = U[E], uW = U[W], uN = U[Nn], uS = U[S], uNE = U[NE],
                             uNW = U[NW], uSE = U[SE], uSW = U[SW];
                const double vP = V[P], vE = V[E], vW = V[W], vN = V[Nn], vS = V[S], vNE = V[NE],
                             vNW = V[NW], vSE = V[SE], vSW = V[SW];
                /* Eq. FDpressure */
                const double pn =
                    -2.0 * pP * (3 * uP * uP + 3 * vP * vP - 2) / 9.0 -
                    pE * (-6 * uE * uE + 6 * uE + 3 * vE * vE - 2) / 18.0 +
                    pW * (6 * uW * uW + 6 * uW - 3 * vW * vW + 2) / 18.0 -
                    pN * (3 * uN * uN - 6 * vN * vN + 6 * vN - 2) / 18.0 +
                    pS * (-3 * uS * uS + 6 * vS * vS + 6 * vS + 2) / 18.0 +
                    pNE * (3 * uNE * uNE + 9 * uNE * vNE - 3 * uNE + 3 * vNE * vNE - 3 * vNE + 1) / 36.0 +
                    pNW * (3 * uNW * uNW - 9 * uNW * vNW + 3 * uNW + 3 * vNW * vNW - 3 * vNW + 1) / 36.0 +
                    pSE * (3 * uSE * uSE - 9 * uSE * vSE - 3 * uSE + 3 * vSE * vSE + 3 * vSE + 1) / 36.0 +
                    pSW * (3 * uSW * uSW + 9 * uSW * vSW + 3 * uSW + 3 * vSW * vSW + 3 * vSW + 1) / 36.0 +
                    k23 * (-pE * uE + pS * vS + pW * uW - pN * vN +
                           (pSW * uSW + pNW * uNW - pNE * uNE - pSE * uSE) / 4.0 +
                           (pSW * vSW - pNW * vNW - pNE * vNE + pSE * vSE) / 4.0);
                /* Eq. FDjx */
                const double pu =
                    pE * (-6 * uE * uE + 6 * uE + 3 * vE * vE - 2) / 18.0 +
                    pW * (6 * uW * uW + 6 * uW - 3 * vW * vW + 2) / 18.0 -
                    pNE * (3 * uNE * uNE + 9 * uNE * vNE - 3 * uNE + 3 * vNE * vNE - 3 * vNE + 1) / 36.0 +
                    pNW * (3 * uNW * uNW - 9 * uNW * vNW + 3 * uNW + 3 * vNW * vNW - 3 * vNW + 1) / 36.0 -
                    pSE * (3 * uSE * uSE - 9 * uSE * vSE - 3 * uSE + 3 * vSE * vSE + 3 * vSE + 1) / 36.0 +
                    pSW * (3 * uSW * uSW + 9 * uSW * vSW + 3 * uSW + 3 * vSW * vSW + 3 * vSW + 1) / 36.0 +
                    k23 * (pE * uE - 3 * pP * uP + pW * uW +
                           (pNE * uNE + pNW * uNW + pSE * uSE + pSW * uSW) / 4.0 +
                           (pNE * vNE - pNW * vNW - pSE * vSE + pSW * vSW) / 4.0);
                /* Eq. FDjy (with the '+' restored before the last term) */
                const double pv =
                    pN * (3 * uN * uN - 6 * vN * vN + 6 * vN - 2) / 18.0 +
                    pS * (-3 * uS * uS + 6 * vS * vS + 6 * vS + 2) / 18.0 -
                    pNE * (3 * uNE * uNE + 9 * uNE * vNE - 3 * uNE + 3 * vNE * vNE - 3 * vNE + 1) / 36.0 -
                    pNW * (3 * uNW * uNW - 9 * uNW * vNW + 3 * uNW + 3 * vNW * vNW - 3 * vNW + 1) / 36.0 +
                    pSE * (3 * uSE * uSE - 9 * uSE * vSE - 3 * uSE + 3 * vSE * vSE + 3 * vSE + 1) / 36.0 +
                    pSW * (3 * uSW * uSW + 9 * uSW * vSW + 3 * uSW + 3 * vSW * vSW + 3 * vSW + 1) / 36.0 +
                    k23 * (pN * vN - 3 * pP * vP + pS * vS +
                           (pNE * uNE - pNW * uNW - pSE * uSE + pSW * uSW) / 4.0 +
                           (pNE * vNE + pNW * vNW + pSE * vSE + pSW * vSW) / 4.0);
                Dn[P] = pn - 1.0;
                Un[P] = pu / pn;
                Vn[P] = pv / pn;
            }
        double *t0 = D, *t1 = U, *t2 = V;
        D = Dn; U = Un; V = Vn;
        Dn = t0; Un = t1; Vn = t2;
    }
#undef IX
    if (D != d) {
        memcpy(d, D, sizeof(double) * N);
        memcpy(u, U, sizeof(double) * N);
        memcpy(v, V, sizeof(double) * N);
    }
    free(buf);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Adjoint of one step. Given the state at t and lambda+ = dL/d(d+, u+) at t+1,
 * accumulate lambda = dL/d(d, u) at t (the caller zeroes it) and the partial
 * derivatives of L with respect to the two scalars a = 2(omega-1)/omega and
 * b = 2/omega - 1 that multiply the odd parts (Eqs. ACM2.0, ACM2.0ccccbb).
 * Reverse-mode chain rule of node_update, serial (scatter into sources).
 * ------------------------------------------------------------------------- */
static void adjoint_step(const lwo_lattice *L, const lwo_geom *G, double omega, double rho0,
                         const double lid[3], const double force[3], int has_force,
                         const double *d, const double *ux, const double *uy, const double *uz,
                         const double *ld_n, const double *lux_n, const double *luy_n,
                         const double *luz_n, double *ld, double *lux, double *luy, double *luz,
                         double *abar, double *bbar) {
    const double a = 2.0 * (omega - 1.0) / omega;
    const double zero[3] = {0.0, 0.0, 0.0};
    double *lu[3] = {lux, luy, luz};
    for (int z = 0; z < G->n[2]; ++z)
        for (int y = 0; y < G->n[1]; ++y)
            for (int xx = 0; xx < G->n[0]; ++xx) {
                const int x[3] = {xx, y, z};
                const long k = ((long)z * G->n[1] + y) * G->n[0] + xx;
                /* forward recompute of rho+, u+ at x */
                double rn, un[3];
                node_update(L, G, omega, omega, rho0, lid, force, has_force, x, d, ux, uy, uz, &rn, un);
                const double lun[3] = {lux_n[k], luy_n[k], luz_n ? luz_n[k] : 0.0};
                /* u+ = m / rho+, rho+ = 1 + d+ */
                double mbar[3], rbar = ld_n[k];
                for (int b = 0; b < 3; ++b) {
                    mbar[b] = lun[b] / rn;
                    rbar -= lun[b] * un[b] / rn;
                }
                double ux_[3];
                load_u(ux, uy, uz, k, ux_);
                const double rx = 1.0 + d[k];
                for (int i = 0; i < L->Q; ++i) {
                    const double fbar = rbar + L->c[i][0] * mbar[0] + L->c[i][1] * mbar[1] +
                                        L->c[i][2] * mbar[2];
                    int above;
                    const long s = source_of(G, x, L->c[i], &above);
                    if (s >= 0) {
                        double us[3];
                        load_u(ux, uy, uz, s, us);
                        const double rs = 1.0 + d[s];
                        /* f = feq(s) + a (feqo(x) - feqo(s)) */
                        ld[s] += fbar * (feq_drho(L, i, us) - a * feqo_drho(L, i, us));
                        ld[k] += fbar * a * feqo_drho(L, i, ux_);
                        for (int b = 0; b < L->D; ++b) {
                            lu[b][s] += fbar * (feq_du(L, i, rs, us, b) - a * feqo_du(L, i, rs, us, b));
                            lu[b][k] += fbar * a * feqo_du(L, i, rx, ux_, b);
                        }
                        *abar += fbar * (feqo(L, i, rx, ux_) - feqo(L, i, rs, us));
                    } else {
                        const int j = L->bb[i];
                        const double *uw = above ? lid : zero;
                        /* f = feq_j(x) + 2a feqo_i(x) + 2b feqo_i(rho0, u_w) */
                        ld[k] += fbar * (feq_drho(L, j, ux_) + 2.0 * a * feqo_drho(L, i, ux_));
                        for (int b = 0; b < L->D; ++b)
                            lu[b][k] += fbar * (feq_du(L, j, rx, ux_, b) + 2.0 * a * feqo_du(L, i, rx, ux_, b));
                        *abar += fbar * 2.0 * feqo(L, i, rx, ux_);
                        *bbar += fbar * 2.0 * feqo(L, i, rho0, uw);
                    }
                    if (has_force) ld[k] += fbar * feqo_drho(L, i, force);
                }
            }
}

/* Gradient of J = 0.5 sum |u(T) - u_target|^2 with respect to the initial
 * state (d0, u0) and nu, by storing all T+1 states and running adjoint_step
 * backwards. Outputs: *loss, g_d/g_ux/g_uy/g_uz (size N each; g_uz NULL for
 * D2Q9), *g_nu. */
int lwo_grad(int Q, int nx, int ny, int nz, double nu, int bc, double rho0, const double *lid,
             const double *force, long T, const double *d0, const double *ux0, const double *uy0,
             const double *uz0, const double *utx, const double *uty, const double *utz,
             double *loss, double *g_d, double *g_ux, double *g_uy, double *g_uz, double *g_nu) {
    lwo_lattice L;
    lwo_geom G;
    if (make_lattice(Q, &L)) return -1;
    if (make_geom(&L, nx, ny, nz, bc, &G)) return -2;
    if (T < 0) return -4;
    const double zero[3] = {0.0, 0.0, 0.0};
    const double *lid_ = lid ? lid : zero;
    const double *frc = force ? force : zero;
    const int has_force = force && (force[0] != 0.0 || force[1] != 0.0 || force[2] != 0.0);
    const double omega = omega_of_nu(nu);
    const long N = (long)nx * ny * nz;
    const int nf = (Q == 19) ? 4 : 3;
    double *S = (double *)malloc(sizeof(double) * N * nf * (T + 1));
    double *lam = (double *)calloc((size_t)N * nf * 2, sizeof(double));
    if (!S || !lam) {
        free(S);
        free(lam);
        return -6;
    }
#define ST(t, f) (S + ((long)(t) * nf + (f)) * N)
    memcpy(ST(0, 0), d0, sizeof(double) * N);
    memcpy(ST(0, 1), ux0, sizeof(double) * N);
    memcpy(ST(0, 2), uy0, sizeof(double) * N);
    if (nf == 4) memcpy(ST(0, 3), uz0, sizeof(double) * N);
    for (long t = 0; t < T; ++t) {
        for (int f = 0; f < nf; ++f) memcpy(ST(t + 1, f), ST(t, f), sizeof(double) * N);
        int rc = lwo_step(Q, nx, ny, nz, nu, bc, rho0, lid_, frc, 1, ST(t + 1, 0), ST(t + 1, 1),
                          ST(t + 1, 2), nf == 4 ? ST(t + 1, 3) : NULL, 0);
        if (rc) {
            free(S);
            free(lam);
            return rc;
        }
    }
    const double *ut[3] = {utx, uty, utz};
    double J = 0.0;
    double *ln = lam, *lc = lam + (long)N * nf; /* lambda at t+1, lambda at t */
    for (long k = 0; k < N; ++k) {
        ln[k] = 0.0;
        for (int b = 0; b < nf - 1; ++b) {
            const double e = ST(T, 1 + b)[k] - ut[b][k];
            J += 0.5 * e * e;
            ln[(long)(1 + b) * N + k] = e;
        }
    }
    double abar = 0.0, bbar = 0.0;
    for (long t = T - 1; t >= 0; --t) {
        memset(lc, 0, sizeof(double) * N * nf);
        adjoint_step(&L, &G, omega, rho0, lid_, frc, has_force, ST(t, 0), ST(t, 1), ST(t, 2),
                     nf == 4 ? ST(t, 3) : NULL, ln, ln + N, ln + 2 * N, nf == 4 ? ln + 3 * N : NULL,
                     lc, lc + N, lc + 2 * N, nf == 4 ? lc + 3 * N : NULL, &abar, &bbar);
        double *tmp = ln;
        ln = lc;
        lc = tmp;
    }
    /* a = 2(omega-1)/omega, b = 2/omega - 1, omega = 2/(6 nu + 1) */
    const double domega_dnu = -12.0 / ((6.0 * nu + 1.0) * (6.0 * nu + 1.0));
    const double da_domega = 2.0 / (omega * omega);
    const double db_domega = -2.0 / (omega * omega);
    *g_nu = (abar * da_domega + bbar * db_domega) * domega_dnu;
    *loss = J;
    memcpy(g_d, ln, sizeof(double) * N);
    memcpy(g_ux, ln + N, sizeof(double) * N);
    memcpy(g_uy, ln + 2 * N, sizeof(double) * N);
    if (nf == 4 && g_uz) memcpy(g_uz, ln + 3 * N, sizeof(double) * N);
#undef ST
    free(S);
    free(lam);
    return 0;
}
