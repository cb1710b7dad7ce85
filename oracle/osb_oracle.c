/*
 * osb_oracle.c -- plain CPU oracle for one explicit time step of the 3D
 * compressible Navier-Stokes equations on a periodic grid, as solved in the
 * Taylor-Green vortex case of OpenSBLI (Jacobs, Jammy & Sandham,
 * arXiv:1609.01277, Section 3.3).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load this library.  It
 * shares no code, header, table or helper with the CUDA library: every
 * coefficient and formula below is restated here from the paper.
 *
 * Style: slow and literal.  Every derivative is written into a full-grid
 * temporary array (the "work array" of Section 2.2/2.4) and the residual is
 * assembled term by term in the order the equations print them.  FP64
 * throughout; build with -ffp-contract=off so no FMA contraction changes the
 * rounding.  OpenMP parallelises only the outer z loop of each sweep.
 *
 * Layout of every state array: structure of arrays, [field][z][y][x], x
 * fastest, fields (rho, rho*u0, rho*u1, rho*u2, rho*E).  Grid points
 * x_i = i*h with h = 2*pi/N per axis; the point x_N is the periodic image of
 * x_0 (Section 2.6), so all stencil indices wrap modulo N.
 *
 * Readings of the paper that this file takes (where the paper is silent):
 *  - RK3 coefficients: the 2-register low-storage scheme with
 *    beta = (1/4, 3/20, 3/5) and alpha = (2/3, 5/12, 3/5) (Section 2.4 only
 *    names the Carpenter-Kennedy low-storage family).
 *  - Viscosity mu = 1 (constant) in both tau and q.
 *  - Initial temperature T = 1, so rho = gamma M^2 p.
 *  - Energy viscous work: form A differentiates the point-wise product
 *    u_i tau_ij (discretely conservative); form B is the product-rule
 *    expansion u_i d_j tau_ij + tau_ij d_j u_i.
 *  - Repeated-direction second derivatives (d_j d_j, and d_i d_i inside
 *    d_j tau_ij) use the second-derivative stencil; mixed ones (a != b) nest
 *    two first-derivative stencils, inner derivative first (Section 2.1.3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_R 6 /* orders 2..12 */

typedef struct {
    int nx, ny, nz;
    int order;      /* even, 2..12 */
    int visc_form;  /* 0 = form A (conservative), 1 = form B (product rule) */
    double Re, Mach, gamma, Pr, dt;
    int nz_domain;  /* points per 2 pi along z when the array is a z-slab of a
                       larger periodic grid (ghost planes included); 0: nz */
} orc_grid;

/* ------------------------------------------------------------------------ */
/* Threads                                                                   */
/* ------------------------------------------------------------------------ */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Central finite-difference weights of order 2r (Section 2.4: arbitrary     */
/* even order, first and second derivatives).                                */
/*   first:  f'_i  ~ (1/h)   sum_{k=1..r} c_k (f_{i+k} - f_{i-k})            */
/*           c_k = (-1)^{k+1} (r!)^2 / (k (r-k)! (r+k)!)                      */
/*   second: f''_i ~ (1/h^2) [ d_0 f_i + sum_{k=1..r} d_k (f_{i+k}+f_{i-k}) ] */
/*           d_k = 2 c_k / k,   d_0 = -2 sum_{k>=1} d_k                       */
/* c[0] is unused (set to 0).  Returns 0, or -1 for an invalid order.        */
/* ------------------------------------------------------------------------ */
static int64_t fact(int n) {
    int64_t f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

int orc_fd_coeffs(int order, double *c, double *d) {
    if (order < 2 || order > 2 * ORC_MAX_R || (order & 1)) return -1;
    int r = order / 2;
    int64_t rf2 = fact(r) * fact(r);
    c[0] = 0.0;
    double dsum = 0.0;
    for (int k = 1; k <= r; ++k) {
        int64_t den = (int64_t)k * fact(r - k) * fact(r + k);
        double ck = (double)rf2 / (double)den;
        if (!(k & 1)) ck = -ck;
        c[k] = ck;
        d[k] = 2.0 * ck / (double)k;
        dsum += d[k];
    }
    d[0] = -2.0 * dsum;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Periodic index helpers                                                    */
/* ------------------------------------------------------------------------ */
static inline int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

static inline size_t at(const orc_grid *g, int x, int y, int z) {
    return ((size_t)z * g->ny + y) * g->nx + x;
}

static inline size_t npts(const orc_grid *g) {
    return (size_t)g->nx * g->ny * g->nz;
}

static double spacing(const orc_grid *g, int axis) {
    int n = axis == 0 ? g->nx : (axis == 1 ? g->ny : (g->nz_domain > 0 ? g->nz_domain : g->nz));
    return 2.0 * M_PI / (double)n;
}

/* out = first derivative of f along axis (0=x, 1=y, 2=z). */
void orc_d1(const orc_grid *g, int axis, const double *f, double *out) {
    double c[ORC_MAX_R + 1], d[ORC_MAX_R + 1];
    orc_fd_coeffs(g->order, c, d);
    int r = g->order / 2;
    double h = spacing(g, axis);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                double s = 0.0;
                for (int k = 1; k <= r; ++k) {
                    double fp, fm;
                    if (axis == 0) {
                        fp = f[at(g, wrap(x + k, g->nx), y, z)];
                        fm = f[at(g, wrap(x - k, g->nx), y, z)];
                    } else if (axis == 1) {
                        fp = f[at(g, x, wrap(y + k, g->ny), z)];
                        fm = f[at(g, x, wrap(y - k, g->ny), z)];
                    } else {
                        fp = f[at(g, x, y, wrap(z + k, g->nz))];
                        fm = f[at(g, x, y, wrap(z - k, g->nz))];
                    }
                    s += c[k] * (fp - fm);
                }
                out[at(g, x, y, z)] = s / h;
            }
}

/* out = second derivative of f along axis (the repeated-index d_a d_a). */
void orc_d2(const orc_grid *g, int axis, const double *f, double *out) {
    double c[ORC_MAX_R + 1], d[ORC_MAX_R + 1];
    orc_fd_coeffs(g->order, c, d);
    int r = g->order / 2;
    double h = spacing(g, axis);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                double s = d[0] * f[at(g, x, y, z)];
                for (int k = 1; k <= r; ++k) {
                    double fp, fm;
                    if (axis == 0) {
                        fp = f[at(g, wrap(x + k, g->nx), y, z)];
                        fm = f[at(g, wrap(x - k, g->nx), y, z)];
                    } else if (axis == 1) {
                        fp = f[at(g, x, wrap(y + k, g->ny), z)];
                        fm = f[at(g, x, wrap(y - k, g->ny), z)];
                    } else {
                        fp = f[at(g, x, y, wrap(z + k, g->nz))];
                        fm = f[at(g, x, y, wrap(z - k, g->nz))];
                    }
                    s += d[k] * (fp + fm);
                }
                out[at(g, x, y, z)] = s / (h * h);
            }
}

/* ------------------------------------------------------------------------ */
/* Point-wise helpers                                                        */
/* ------------------------------------------------------------------------ */
static double *alloc(size_t n) { return (double *)calloc(n, sizeof(double)); }

/* dst[p] += a * x[p] */
static void axpy(size_t n, double a, const double *x, double *dst) {
#pragma omp parallel for schedule(static)
    for (long p = 0; p < (long)n; ++p) dst[p] += a * x[p];
}

/* dst[p] += a * x[p] * y[p] */
static void axypz(size_t n, double a, const double *x, const double *y, double *dst) {
#pragma omp parallel for schedule(static)
    for (long p = 0; p < (long)n; ++p) dst[p] += a * x[p] * y[p];
}

/* dst[p] = x[p] * y[p] */
static void mul(size_t n, const double *x, const double *y, double *dst) {
#pragma omp parallel for schedule(static)
    for (long p = 0; p < (long)n; ++p) dst[p] = x[p] * y[p];
}

/* Primitive variables from the conserved state.
 * u_i = (rho u_i)/rho; rho E = p/(gamma-1) + (1/2) rho u_j u_j (Eq. for rhoE)
 * so p = (gamma-1)(rho E - (1/2) rho u_j u_j); equation of state
 * p = rho T / (gamma M^2)  =>  T = gamma M^2 p / rho. */
void orc_primitives(const orc_grid *g, const double *Q, double *u /*3N*/,
                    double *p, double *T) {
    size_t n = npts(g);
    double gm1 = g->gamma - 1.0;
    double gM2 = g->gamma * g->Mach * g->Mach;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)n; ++i) {
        double rho = Q[i];
        double u0 = Q[n + i] / rho, u1 = Q[2 * n + i] / rho, u2 = Q[3 * n + i] / rho;
        u[i] = u0;
        u[n + i] = u1;
        u[2 * n + i] = u2;
        double ke = 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2);
        double pp = gm1 * (Q[4 * n + i] - ke);
        p[i] = pp;
        T[i] = gM2 * pp / rho;
    }
}

/* ------------------------------------------------------------------------ */
/* Residual R(Q) = dQ/dt of the semi-discrete equations (Section 3.3).       */
/*                                                                           */
/*  mass:     d rho/dt   = - Skew(rho)                                       */
/*  momentum: d rhou_i/dt = - Skew(rho u_i) - d_i p + d_j tau_ij             */
/*  energy:   d rhoE/dt  = - Skew(rho E) - d_j (u_j p) + d_j q_j             */
/*                          + d_j (u_i tau_ij)                               */
/*  Skew(rho phi) = 1/2 [ d_j(rho phi u_j) + u_j d_j(rho phi)                */
/*                        + rho phi d_j u_j ]        (skew-symmetric form)    */
/*  tau_ij = (1/Re)(d_j u_i + d_i u_j - 2/3 delta_ij d_k u_k)                */
/*  q_j    = mu/((gamma-1) M^2 Pr Re) d_j T,  mu = 1                          */
/* ------------------------------------------------------------------------ */
int orc_residual(const orc_grid *g, const double *Q, double *R) {
    size_t n = npts(g);
    double *u = alloc(3 * n), *p = alloc(n), *T = alloc(n);
    double *G = alloc(9 * n);  /* G[i*3+j] = d_j u_i, first-derivative stencil */
    double *t1 = alloc(n), *t2 = alloc(n), *t3 = alloc(n);
    double *divu = alloc(n);
    if (!u || !p || !T || !G || !t1 || !t2 || !t3 || !divu) {
        free(u); free(p); free(T); free(G); free(t1); free(t2); free(t3); free(divu);
        return -1;
    }
    double inv_re = 1.0 / g->Re;
    double kappa = 1.0 / ((g->gamma - 1.0) * g->Mach * g->Mach * g->Pr * g->Re);

    orc_primitives(g, Q, u, p, T);
    memset(R, 0, 5 * n * sizeof(double));

    /* velocity gradient and divergence */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) orc_d1(g, j, u + i * n, G + (i * 3 + j) * n);
    for (size_t q = 0; q < n; ++q) divu[q] = G[0 * n + q] + G[4 * n + q] + G[8 * n + q];

    /* --- convective terms, skew-symmetric, for each conserved field ------ */
    for (int m = 0; m < 5; ++m) {
        const double *a = Q + m * n; /* rho*phi with phi = 1, u_i, E */
        double *Rm = R + m * n;
        for (int j = 0; j < 3; ++j) {
            const double *uj = u + j * n;
            mul(n, a, uj, t1);           /* rho phi u_j            */
            orc_d1(g, j, t1, t2);        /* d_j (rho phi u_j)      */
            axpy(n, -0.5, t2, Rm);
            orc_d1(g, j, a, t2);         /* d_j (rho phi)          */
            axypz(n, -0.5, uj, t2, Rm);  /* u_j d_j (rho phi)      */
            axypz(n, -0.5, a, G + (j * 3 + j) * n, Rm); /* rho phi d_j u_j */
        }
    }

    /* --- pressure terms ----------------------------------------------- */
    for (int i = 0; i < 3; ++i) {
        orc_d1(g, i, p, t1);                 /* d_i p */
        axpy(n, -1.0, t1, R + (1 + i) * n);
    }
    for (int j = 0; j < 3; ++j) {
        mul(n, u + j * n, p, t1);            /* u_j p */
        orc_d1(g, j, t1, t2);                /* d_j (u_j p) */
        axpy(n, -1.0, t2, R + 4 * n);
    }

    /* --- d_j tau_ij, expanded to second derivatives ---------------------
     * d_j tau_ij = (1/Re) sum_j [ d_j d_j u_i + d_j d_i u_j
     *                             - 2/3 delta_ij sum_k d_i d_k u_k ]
     * repeated direction -> second-derivative stencil, mixed -> nested d1.
     * dtau[i] keeps the sum for the form-B viscous work. */
    double *dtau = alloc(3 * n);
    if (!dtau) { free(u); free(p); free(T); free(G); free(t1); free(t2); free(t3); free(divu); return -1; }
    for (int i = 0; i < 3; ++i) {
        double *Di = dtau + i * n;
        for (int j = 0; j < 3; ++j) {
            /* d_j d_j u_i */
            orc_d2(g, j, u + i * n, t1);
            axpy(n, inv_re, t1, Di);
            /* d_j d_i u_j */
            if (j == i) {
                orc_d2(g, i, u + i * n, t1);
            } else {
                orc_d1(g, j, G + (j * 3 + i) * n, t1); /* d_j (d_i u_j) */
            }
            axpy(n, inv_re, t1, Di);
        }
        /* -2/3 d_i (d_k u_k) for the j = i term */
        for (int k = 0; k < 3; ++k) {
            if (k == i) {
                orc_d2(g, i, u + i * n, t1);
            } else {
                orc_d1(g, i, G + (k * 3 + k) * n, t1); /* d_i (d_k u_k) */
            }
            axpy(n, -2.0 / 3.0 * inv_re, t1, Di);
        }
        axpy(n, 1.0, Di, R + (1 + i) * n);
    }

    /* --- heat flux: d_j q_j = kappa sum_j d_j d_j T ----------------------- */
    for (int j = 0; j < 3; ++j) {
        orc_d2(g, j, T, t1);
        axpy(n, kappa, t1, R + 4 * n);
    }

    /* --- viscous work d_j (u_i tau_ij) ----------------------------------- */
    if (g->visc_form == 0) {
        /* form A: tau_ij at each point from first derivatives, then d_j of
         * the point-wise product u_i tau_ij */
        for (int j = 0; j < 3; ++j) {
            memset(t1, 0, n * sizeof(double));
            for (int i = 0; i < 3; ++i) {
                const double *dj_ui = G + (i * 3 + j) * n;
                const double *di_uj = G + (j * 3 + i) * n;
                const double *ui = u + i * n;
#pragma omp parallel for schedule(static)
                for (long q = 0; q < (long)n; ++q) {
                    double tau = dj_ui[q] + di_uj[q];
                    if (i == j) tau -= 2.0 / 3.0 * divu[q];
                    tau *= inv_re;
                    t1[q] += ui[q] * tau;
                }
            }
            orc_d1(g, j, t1, t2);
            axpy(n, 1.0, t2, R + 4 * n);
        }
    } else {
        /* form B: u_i d_j tau_ij + tau_ij d_j u_i */
        for (int i = 0; i < 3; ++i) axypz(n, 1.0, u + i * n, dtau + i * n, R + 4 * n);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                const double *dj_ui = G + (i * 3 + j) * n;
                const double *di_uj = G + (j * 3 + i) * n;
#pragma omp parallel for schedule(static)
                for (long q = 0; q < (long)n; ++q) {
                    double tau = dj_ui[q] + di_uj[q];
                    if (i == j) tau -= 2.0 / 3.0 * divu[q];
                    tau *= inv_re;
                    R[4 * n + q] += tau * dj_ui[q];
                }
            }
    }

    free(u); free(p); free(T); free(G); free(t1); free(t2); free(t3); free(divu); free(dtau);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Low-storage third-order Runge-Kutta (Section 2.4), two registers.          */
/*   q_0 = U_0 = Q^n                                                          */
/*   stage k = 1..3:  R = R(q_{k-1});  q_k = U_{k-1} + alpha_k dt R;          */
/*                    U_k = U_{k-1} + beta_k dt R                              */
/*   Q^{n+1} = U_3                                                             */
/* ------------------------------------------------------------------------ */
static const double RK_ALPHA[3] = {2.0 / 3.0, 5.0 / 12.0, 3.0 / 5.0};
static const double RK_BETA[3] = {1.0 / 4.0, 3.0 / 20.0, 3.0 / 5.0};

void orc_rk3_coeffs(double *alpha, double *beta) {
    for (int k = 0; k < 3; ++k) {
        alpha[k] = RK_ALPHA[k];
        beta[k] = RK_BETA[k];
    }
}

typedef int (*orc_rhs_fn)(void *ctx, const double *y, double *r);

/* Generic driver: advances y (length n) by nsteps steps of size dt. */
static int lsrk3(size_t n, double *y, int nsteps, double dt, orc_rhs_fn rhs, void *ctx) {
    double *q = alloc(n), *R = alloc(n);
    if (!q || !R) { free(q); free(R); return -1; }
    for (int s = 0; s < nsteps; ++s) {
        memcpy(q, y, n * sizeof(double));           /* q_0 = U_0 = y */
        for (int k = 0; k < 3; ++k) {
            if (rhs(ctx, q, R)) { free(q); free(R); return -1; }
            double a = RK_ALPHA[k] * dt, b = RK_BETA[k] * dt;
#pragma omp parallel for schedule(static)
            for (long i = 0; i < (long)n; ++i) {
                q[i] = y[i] + a * R[i];
                y[i] = y[i] + b * R[i];
            }
        }
    }
    free(q); free(R);
    return 0;
}

/* Forward Euler (Section 2.4 offers it beside the RK3 scheme):
 * y^{n+1} = y^n + dt R(y^n). */
static int euler(size_t n, double *y, int nsteps, double dt, orc_rhs_fn rhs, void *ctx) {
    double *R = alloc(n);
    if (!R) return -1;
    for (int s = 0; s < nsteps; ++s) {
        if (rhs(ctx, y, R)) { free(R); return -1; }
#pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)n; ++i) y[i] = y[i] + dt * R[i];
    }
    free(R);
    return 0;
}

static int ns_rhs(void *ctx, const double *y, double *r) {
    return orc_residual((const orc_grid *)ctx, y, r);
}

/* Advance the conserved state Q in place by nsteps forward-Euler steps. */
int orc_euler_step(const orc_grid *g, double *Q, int nsteps) {
    return euler(5 * npts(g), Q, nsteps, g->dt, ns_rhs, (void *)g);
}

/* Advance the conserved state Q (5 fields) in place by nsteps RK3 steps. */
int orc_rk3_step(const orc_grid *g, double *Q, int nsteps) {
    return lsrk3(5 * npts(g), Q, nsteps, g->dt, ns_rhs, (void *)g);
}

/* Same driver on the linear system dy_i/dt = lambda_i y_i (real lambda):
 * lets the tests check the scheme's order and stability polynomial. */
typedef struct { size_t n; const double *lam; } lin_ctx;
static int lin_rhs(void *ctx, const double *y, double *r) {
    const lin_ctx *c = (const lin_ctx *)ctx;
    for (size_t i = 0; i < c->n; ++i) r[i] = c->lam[i] * y[i];
    return 0;
}

int orc_rk3_linear(size_t n, const double *lam, double *y, int nsteps, double dt) {
    lin_ctx c = {n, lam};
    return lsrk3(n, y, nsteps, dt, lin_rhs, &c);
}

int orc_euler_linear(size_t n, const double *lam, double *y, int nsteps, double dt) {
    lin_ctx c = {n, lam};
    return euler(n, y, nsteps, dt, lin_rhs, &c);
}

/* ------------------------------------------------------------------------ */
/* Scalar advection-diffusion on the periodic box, the equation of the       */
/* Section 3.1 wave test (k = 0, S = 0) and of the Section 3.2 manufactured-  */
/* solution test:                                                            */
/*   d phi/dt + d_j(phi a_j - k d_j phi) + S = 0,  a_j and k constant,        */
/* so  d phi/dt = - sum_j a_j D_j phi + k sum_j L_j phi - S,  with the first- */
/* and second-derivative stencils of the grid's order.  An axis with one     */
/* point carries no derivative (the 1D and 2D tests are 3D grids with        */
/* unit extents).  S may be NULL (no source).                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_grid *g;
    double a[3], k;
    const double *S;
    double *w;
} scalar_ctx;

static int scalar_rhs(void *ctx, const double *y, double *r) {
    const scalar_ctx *c = (const scalar_ctx *)ctx;
    const size_t n = npts(c->g);
    const int dims[3] = {c->g->nx, c->g->ny, c->g->nz};
    for (size_t i = 0; i < n; ++i) r[i] = 0.0;
    for (int axis = 0; axis < 3; ++axis) {
        if (dims[axis] < 2) continue;
        if (c->a[axis] != 0.0) {
            orc_d1(c->g, axis, y, c->w);
            for (size_t i = 0; i < n; ++i) r[i] -= c->a[axis] * c->w[i];
        }
        if (c->k != 0.0) {
            orc_d2(c->g, axis, y, c->w);
            for (size_t i = 0; i < n; ++i) r[i] += c->k * c->w[i];
        }
    }
    if (c->S)
        for (size_t i = 0; i < n; ++i) r[i] -= c->S[i];
    return 0;
}

/* Advance phi (one field on the grid) by nsteps RK3 steps of g->dt. */
int orc_scalar_rk3(const orc_grid *g, const double *a, double k, const double *S, double *phi, int nsteps) {
    scalar_ctx c;
    c.g = g;
    c.a[0] = a[0], c.a[1] = a[1], c.a[2] = a[2];
    c.k = k;
    c.S = S;
    c.w = alloc(npts(g));
    if (!c.w) return -1;
    int rc = lsrk3(npts(g), phi, nsteps, g->dt, scalar_rhs, &c);
    free(c.w);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Taylor-Green vortex initial state (Section 3.3), L = 1:                   */
/*   u0 = sin x cos y cos z,  u1 = -cos x sin y cos z,  u2 = 0               */
/*   p  = 1/(gamma M^2) + (1/16)(cos 2x + cos 2y)(2 + cos 2z)                 */
/* with T = 1, so rho = gamma M^2 p.  Optional perturbation: u_i +=           */
/* amp * noise[i][point] at fixed rho and p (noise supplied by the caller).   */
/* ------------------------------------------------------------------------ */
void orc_tgv_init(const orc_grid *g, const double *noise, double amp, double *Q) {
    size_t n = npts(g);
    double gM2 = g->gamma * g->Mach * g->Mach;
    double hx = spacing(g, 0), hy = spacing(g, 1), hz = spacing(g, 2);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t i = at(g, x, y, z);
                double X = x * hx, Y = y * hy, Z = z * hz;
                double u0 = sin(X) * cos(Y) * cos(Z);
                double u1 = -cos(X) * sin(Y) * cos(Z);
                double u2 = 0.0;
                double p = 1.0 / gM2 + (cos(2.0 * X) + cos(2.0 * Y)) * (2.0 + cos(2.0 * Z)) / 16.0;
                double rho = gM2 * p; /* T = 1 */
                if (noise) {
                    u0 += amp * noise[i];
                    u1 += amp * noise[n + i];
                    u2 += amp * noise[2 * n + i];
                }
                Q[i] = rho;
                Q[n + i] = rho * u0;
                Q[2 * n + i] = rho * u1;
                Q[3 * n + i] = rho * u2;
                Q[4 * n + i] = p / (g->gamma - 1.0) + 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2);
            }
}

/* ------------------------------------------------------------------------ */
/* Diagnostics (Section 3.3): grid means, with rho_ref = 1.                  */
/*  out[0] = E_k  = <(1/2) rho u_j u_j>                                      */
/*  out[1] = enstrophy = <(1/2) rho (eps_ijk d_j u_k)^2>, d_j = first-deriv.  */
/*  out[2..6] = <rho>, <rho u_0>, <rho u_1>, <rho u_2>, <rho E>              */
/*  out[7] = number of points with a non-finite conserved value              */
/*  out[8] = max CFL = dt * max_points sum_j (|u_j| + c)/h_j, c^2 = gamma p/rho */
/* ------------------------------------------------------------------------ */
int orc_diagnostics(const orc_grid *g, const double *Q, double *out) {
    size_t n = npts(g);
    double *u = alloc(3 * n), *p = alloc(n), *T = alloc(n), *G = alloc(9 * n);
    if (!u || !p || !T || !G) { free(u); free(p); free(T); free(G); return -1; }
    orc_primitives(g, Q, u, p, T);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) orc_d1(g, j, u + i * n, G + (i * 3 + j) * n);
    double h[3] = {spacing(g, 0), spacing(g, 1), spacing(g, 2)};
    double ke = 0, ens = 0, tot[5] = {0, 0, 0, 0, 0}, nonfinite = 0, cfl = 0;
    for (size_t q = 0; q < n; ++q) {
        double rho = Q[q];
        double uu = 0.0;
        for (int j = 0; j < 3; ++j) uu += u[j * n + q] * u[j * n + q];
        ke += 0.5 * rho * uu;
        /* omega_i = eps_ijk d_j u_k */
        double w0 = G[(2 * 3 + 1) * n + q] - G[(1 * 3 + 2) * n + q]; /* d_1 u_2 - d_2 u_1 */
        double w1 = G[(0 * 3 + 2) * n + q] - G[(2 * 3 + 0) * n + q]; /* d_2 u_0 - d_0 u_2 */
        double w2 = G[(1 * 3 + 0) * n + q] - G[(0 * 3 + 1) * n + q]; /* d_0 u_1 - d_1 u_0 */
        ens += 0.5 * rho * (w0 * w0 + w1 * w1 + w2 * w2);
        int bad = 0;
        for (int m = 0; m < 5; ++m) {
            tot[m] += Q[m * n + q];
            if (!isfinite(Q[m * n + q])) bad = 1;
        }
        nonfinite += bad;
        double c = sqrt(g->gamma * p[q] / rho);
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += (fabs(u[j * n + q]) + c) / h[j];
        if (s * g->dt > cfl) cfl = s * g->dt;
    }
    out[0] = ke / (double)n;
    out[1] = ens / (double)n;
    for (int m = 0; m < 5; ++m) out[2 + m] = tot[m] / (double)n;
    out[7] = nonfinite;
    out[8] = cfl;
    free(u); free(p); free(T); free(G);
    return 0;
}
