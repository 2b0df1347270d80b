/*
 * swe_oracle.c -- plain, slow FP64 CPU oracle of one explicit 2D MacCormack
 * predictor-corrector time step of the shallow-water equations, the method of
 * Seitz, Kennedy, Ransom, Younis and Owens, "A GPU Implementation for
 * Two-Dimensional Shallow Water Modeling" (2013), Sec. 1.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the yardstick the CUDA path is
 * checked against.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may build, load or call it.  It shares no code, header,
 * table or helper with the CUDA library and must never be linked into it.
 *
 * What the paper fixes (Sec. 1): the unknowns are the free-surface elevation
 * and the two depth-averaged velocities of every cell; the scheme is an
 * explicit 2D predictor/corrector MacCormack method; one time step is a chain
 * of 16 dependent sub-steps, each independent per cell, each reading neighbour
 * values written by the previous one.  Sec. 3.1 adds that the step size is
 * variable (a CFL-type serial reduction).  Sec. 6.2 says the original code had
 * no wet/dry treatment.  Everything else (the equations, the one-sided
 * differences, boundary conditions, friction law, time-step formula, drying,
 * dissipation) is deferred by the paper to Ransom's thesis, which is not
 * available; the readings adopted here are the standard 2D MacCormack form on
 * the non-conservative elevation/velocity equations
 *
 *     eta_t + (h u)_x + (h v)_y = 0
 *     u_t + u u_x + v u_y + g eta_x = - g n^2 u |U| / h^(4/3)
 *     v_t + u v_x + v v_y + g eta_y = - g n^2 v |U| / h^(4/3)
 *
 * with h = eta - z.  The step is written as the 16 sub-steps S1..S16 below,
 * each one a full-grid pass, run in order; no pass is fused with another.
 *
 * Layout: caller arrays are ny*nx doubles, row-major, x (index i) fastest,
 * cell (i,j) at index j*nx+i.  Internally every level keeps a one-cell ghost
 * ring, index (j+1)*(nx+2)+(i+1); corners of the ring are never read.
 *
 * Rounding: IEEE binary64, round to nearest; build with -ffp-contract=off and
 * without -ffast-math so no fused multiply-add is formed.  The x term is
 * always added before the y term.  Every sum over cells is taken per row in
 * increasing i and then over rows in increasing j, so the result does not
 * depend on the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { BC_WALL = 0, BC_INFLOW = 1, BC_OUTFLOW = 2 };
enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };
enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NONFINITE = 3 };

/* Dissipation switch denominator guard (metres); keeps nu finite on dry rows. */
#define NU_TINY 1e-12

typedef struct {
    int32_t nx, ny;
    double dx, dy;      /* cell sizes, m */
    double g;           /* gravity, m/s^2 */
    double cfl;         /* Courant number of the time-step rule */
    double h_dry;       /* wet iff h > h_dry, m */
    double dt_max;      /* upper bound of the time step, s */
    double kappa;       /* artificial dissipation coefficient, 0 = off */
    double manning_n;   /* uniform Manning n when no per-cell field is given */
    int32_t bc[4];      /* W, E, S, N: BC_WALL / BC_INFLOW / BC_OUTFLOW */
    double q_in[4];     /* inflow discharge per unit width INTO the domain, m^2/s */
    int32_t dir_cycle;  /* predictor direction schedule, see step_dirs() */
    int32_t friction;   /* 0: point-implicit Manning (the reading used throughout); 1: explicit */
    int32_t dissipation;/* 0: S15 as below (kappa); 1: the TVD-MacCormack term (kappa ignored) */
} orc_params;

/* ------------------------------------------------------------------ */
/* Work arrays                                                         */
/* ------------------------------------------------------------------ */
typedef struct {
    int nx, ny, W;
    double *z, *n2;
    /* level n */
    double *eta, *u, *v, *h; unsigned char *wet;
    double *qx, *qy, *fx, *fy, *C;
    /* predicted level (*) */
    double *es, *us, *vs, *hs; unsigned char *wets;
    double *qxs, *qys, *fxs, *fys, *Cs;
    /* corrected level (**) */
    double *ess, *uss, *vss;
    /* new level n+1 */
    double *e1, *u1, *v1;
    /* dissipation switches */
    double *nux, *nuy;
    /* per-row partial tallies */
    double *row_a, *row_b;
} work;

#define G(i, j) ((size_t)((j) + 1) * (size_t)w->W + (size_t)((i) + 1))
/* x-face i+1/2, i in [-1, nx-1], of row j */
#define FX(i, j) ((size_t)(j) * (size_t)(w->nx + 1) + (size_t)((i) + 1))
/* y-face j+1/2, j in [-1, ny-1], of column i */
#define FY(i, j) ((size_t)((j) + 1) * (size_t)w->nx + (size_t)(i))

static void work_free(work* w) {
    void* ptrs[] = {w->z, w->n2, w->eta, w->u, w->v, w->h, w->wet, w->qx, w->qy,
                    w->fx, w->fy, w->C, w->es, w->us, w->vs, w->hs, w->wets,
                    w->qxs, w->qys, w->fxs, w->fys, w->Cs, w->ess, w->uss,
                    w->vss, w->e1, w->u1, w->v1, w->nux, w->nuy, w->row_a, w->row_b};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    memset(w, 0, sizeof(*w));
}

static int work_alloc(work* w, int nx, int ny) {
    memset(w, 0, sizeof(*w));
    w->nx = nx; w->ny = ny; w->W = nx + 2;
    size_t nc = (size_t)(nx + 2) * (size_t)(ny + 2);
    size_t nfx = (size_t)(nx + 1) * (size_t)ny;
    size_t nfy = (size_t)nx * (size_t)(ny + 1);
#define A(p, n) do { (p) = calloc((n), sizeof(*(p))); if (!(p)) { work_free(w); return 0; } } while (0)
    A(w->z, nc); A(w->n2, nc);
    A(w->eta, nc); A(w->u, nc); A(w->v, nc); A(w->h, nc); A(w->wet, nc);
    A(w->qx, nc); A(w->qy, nc); A(w->fx, nfx); A(w->fy, nfy); A(w->C, nc);
    A(w->es, nc); A(w->us, nc); A(w->vs, nc); A(w->hs, nc); A(w->wets, nc);
    A(w->qxs, nc); A(w->qys, nc); A(w->fxs, nfx); A(w->fys, nfy); A(w->Cs, nc);
    A(w->ess, nc); A(w->uss, nc); A(w->vss, nc);
    A(w->e1, nc); A(w->u1, nc); A(w->v1, nc);
    A(w->nux, nc); A(w->nuy, nc);
    A(w->row_a, (size_t)ny); A(w->row_b, (size_t)ny);
#undef A
    return 1;
}

/* Predictor one-sided direction per axis for step index k: +1 = forward
 * difference (F), -1 = backward (B); the corrector takes the opposite.
 * dir_cycle bit 0: flip both directions on odd steps (alternating FF/BB);
 * bit 1: x starts backward; bit 2: y starts backward. */
static void step_dirs(int32_t dir_cycle, int64_t k, int* sx, int* sy) {
    int ax = (dir_cycle & 2) ? -1 : +1;
    int ay = (dir_cycle & 4) ? -1 : +1;
    if ((dir_cycle & 1) && (k & 1)) { ax = -ax; ay = -ay; }
    *sx = ax; *sy = ay;
}

/* Elevation of a neighbour as seen by the pressure term of cell `self`:
 * a dry neighbour whose bed lies above the water surface of `self` acts
 * as a wall (zero gradient); otherwise its real surface is used. */
static double eta_seen(double eta_nb, double z_nb, unsigned char wet_nb, double eta_self) {
    return (!wet_nb && z_nb > eta_self) ? eta_self : eta_nb;
}

/* ------------------------------------------------------------------ */
/* S3 / S9: ghost ring from the boundary conditions                    */
/* ------------------------------------------------------------------ */
/* Ghost of every kind copies the adjacent interior elevation, bed and depth.
 * WALL: normal velocity reflected, tangential copied (free slip).
 * INFLOW: normal velocity = q_in / max(h_in, h_dry) pointing into the domain,
 *         tangential 0.  OUTFLOW: every field copied (transmissive). */
static void fill_ghosts(const orc_params* p, work* w, double* eta, double* u, double* v,
                        double* h, unsigned char* wet) {
    const int nx = w->nx, ny = w->ny;
    for (int j = 0; j < ny; ++j) {
        for (int side = SIDE_W; side <= SIDE_E; ++side) {
            int ii = (side == SIDE_W) ? 0 : nx - 1;
            int ig = (side == SIDE_W) ? -1 : nx;
            double sgn = (side == SIDE_W) ? 1.0 : -1.0;
            size_t a = G(ii, j), b = G(ig, j);
            eta[b] = eta[a]; h[b] = h[a]; wet[b] = wet[a];
            switch (p->bc[side]) {
            case BC_WALL:   u[b] = -u[a]; v[b] = v[a]; break;
            case BC_INFLOW: u[b] = sgn * p->q_in[side] / fmax(h[a], p->h_dry); v[b] = 0.0; break;
            default:        u[b] = u[a]; v[b] = v[a]; break;
            }
        }
    }
    for (int i = 0; i < nx; ++i) {
        for (int side = SIDE_S; side <= SIDE_N; ++side) {
            int jj = (side == SIDE_S) ? 0 : ny - 1;
            int jg = (side == SIDE_S) ? -1 : ny;
            double sgn = (side == SIDE_S) ? 1.0 : -1.0;
            size_t a = G(i, jj), b = G(i, jg);
            eta[b] = eta[a]; h[b] = h[a]; wet[b] = wet[a];
            switch (p->bc[side]) {
            case BC_WALL:   v[b] = -v[a]; u[b] = u[a]; break;
            case BC_INFLOW: v[b] = sgn * p->q_in[side] / fmax(h[a], p->h_dry); u[b] = 0.0; break;
            default:        u[b] = u[a]; v[b] = v[a]; break;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* S4 / S10: continuity fluxes h*u, h*v and the face fluxes            */
/* ------------------------------------------------------------------ */
/* dir = +1: face i+1/2 carries the flux of cell i+1 (so the update is a
 * forward difference); dir = -1: it carries the flux of cell i.  Boundary
 * faces: WALL 0, INFLOW the prescribed discharge, OUTFLOW the flux of the
 * adjacent interior cell. */
static void fluxes(const orc_params* p, work* w, const double* h, const double* u,
                   const double* v, double* qx, double* qy, double* fx, double* fy,
                   int sx, int sy) {
    const int nx = w->nx, ny = w->ny;
    #pragma omp parallel for schedule(static)
    for (int j = -1; j <= ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            int ghost_i = (i < 0 || i >= nx), ghost_j = (j < 0 || j >= ny);
            if (ghost_i && ghost_j) continue;  /* corners are never used */
            size_t c = G(i, j);
            qx[c] = h[c] * u[c];
            qy[c] = h[c] * v[c];
        }
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = -1; i < nx; ++i) {
            double f;
            if (i == -1 || i == nx - 1) {
                int side = (i == -1) ? SIDE_W : SIDE_E;
                int inner = (i == -1) ? 0 : nx - 1;
                if (p->bc[side] == BC_WALL) f = 0.0;
                else if (p->bc[side] == BC_INFLOW) f = (side == SIDE_W) ? p->q_in[side] : -p->q_in[side];
                else f = qx[G(inner, j)];
            } else {
                f = (sx > 0) ? qx[G(i + 1, j)] : qx[G(i, j)];
            }
            fx[FX(i, j)] = f;
        }
    #pragma omp parallel for schedule(static)
    for (int j = -1; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double f;
            if (j == -1 || j == ny - 1) {
                int side = (j == -1) ? SIDE_S : SIDE_N;
                int inner = (j == -1) ? 0 : ny - 1;
                if (p->bc[side] == BC_WALL) f = 0.0;
                else if (p->bc[side] == BC_INFLOW) f = (side == SIDE_S) ? p->q_in[side] : -p->q_in[side];
                else f = qy[G(i, inner)];
            } else {
                f = (sy > 0) ? qy[G(i, j + 1)] : qy[G(i, j)];
            }
            fy[FY(i, j)] = f;
        }
}

/* S5 / S11: continuity, eta_out = eta_n - dt * (div_x + div_y) */
static void continuity(work* w, double dt, double dx, double dy, const double* eta_n,
                       const double* fx, const double* fy, double* eta_out) {
    const int nx = w->nx, ny = w->ny;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double divx = (fx[FX(i, j)] - fx[FX(i - 1, j)]) / dx;
            double divy = (fy[FY(i, j)] - fy[FY(i, j - 1)]) / dy;
            eta_out[G(i, j)] = eta_n[G(i, j)] - dt * (divx + divy);
        }
}

/* S6 / S12: point-implicit Manning coefficient C = g n^2 |U| / h^(4/3), wet cells only */
static void friction(const orc_params* p, work* w, const double* h, const unsigned char* wet,
                     const double* u, const double* v, double* C) {
    const int nx = w->nx, ny = w->ny;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            C[c] = wet[c] ? p->g * w->n2[c] * sqrt(u[c] * u[c] + v[c] * v[c]) / pow(h[c], 4.0 / 3.0)
                          : 0.0;
        }
}

/* S7 / S13: momentum.  The differenced state (eta, u, v, wet) is the
 * predictor input for S7 and the predicted state for S13; u_n, v_n are
 * always the level-n velocities.  out = (vel_n - dt*A) / (1 + dt*C), or with
 * explicit friction (the ablation) out = vel_n - dt*A - dt*C*vel, C and vel
 * those of the differenced state. */
static void momentum(const orc_params* p, work* w, double dt, int sx, int sy,
                     const double* eta, const double* u, const double* v,
                     const unsigned char* wet, const double* C,
                     const double* u_n, const double* v_n, double* u_out, double* v_out) {
    const int nx = w->nx, ny = w->ny;
    const double* z = w->z;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            size_t xn = (sx > 0) ? G(i + 1, j) : G(i - 1, j);
            size_t yn = (sy > 0) ? G(i, j + 1) : G(i, j - 1);
            double dux, dvx, dex, duy, dvy, dey;
            double ex = eta_seen(eta[xn], z[xn], wet[xn], eta[c]);
            double ey = eta_seen(eta[yn], z[yn], wet[yn], eta[c]);
            if (sx > 0) { dux = u[xn] - u[c]; dvx = v[xn] - v[c]; dex = ex - eta[c]; }
            else        { dux = u[c] - u[xn]; dvx = v[c] - v[xn]; dex = eta[c] - ex; }
            if (sy > 0) { duy = u[yn] - u[c]; dvy = v[yn] - v[c]; dey = ey - eta[c]; }
            else        { duy = u[c] - u[yn]; dvy = v[c] - v[yn]; dey = eta[c] - ey; }
            double Au = u[c] * dux / p->dx + v[c] * duy / p->dy + p->g * dex / p->dx;
            double Av = u[c] * dvx / p->dx + v[c] * dvy / p->dy + p->g * dey / p->dy;
            if (p->friction == 1) {
                u_out[c] = (u_n[c] - dt * Au) - dt * C[c] * u[c];
                v_out[c] = (v_n[c] - dt * Av) - dt * C[c] * v[c];
            } else {
                double den = 1.0 + dt * C[c];
                u_out[c] = (u_n[c] - dt * Au) / den;
                v_out[c] = (v_n[c] - dt * Av) / den;
            }
        }
}

/* S8 / S16: wet/dry fix.  A negative depth is clamped to zero (eta = z) and
 * the added water is tallied per row in row_acc; a cell with h <= h_dry gets
 * zero velocity.  Writes h and wet of the fixed level. */
static void wetdry_fix(const orc_params* p, work* w, double* eta, double* u, double* v,
                       double* h, unsigned char* wet, double* row_acc) {
    const int nx = w->nx, ny = w->ny;
    const double cell_area = p->dx * p->dy;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        double acc = 0.0;
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            double d = eta[c] - w->z[c];
            if (d < 0.0) { acc += -d * cell_area; eta[c] = w->z[c]; d = 0.0; }
            if (d <= p->h_dry) { u[c] = 0.0; v[c] = 0.0; }
            h[c] = d;
            wet[c] = d > p->h_dry;
        }
        row_acc[j] = acc;
    }
}

static double sum_rows(const double* r, int ny) {
    double s = 0.0;
    for (int j = 0; j < ny; ++j) s += r[j];
    return s;
}

/* S1: depth and wet mask of the level-n state */
static void depth_mask(const orc_params* p, work* w) {
    const int nx = w->nx, ny = w->ny;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            w->h[c] = w->eta[c] - w->z[c];
            w->wet[c] = w->h[c] > p->h_dry;
        }
}

/* S2: CFL time step from the level-n state.  Largest over wet cells of
 * (|u| + sqrt(g h))/dx + (|v| + sqrt(g h))/dy, then dt = cfl / that,
 * capped at dt_max; dt_max when no cell is wet. */
static double cfl_dt(const orc_params* p, work* w) {
    const int nx = w->nx, ny = w->ny;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        double m = 0.0;
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            if (!w->wet[c]) continue;
            double cel = sqrt(p->g * w->h[c]);
            double s = (fabs(w->u[c]) + cel) / p->dx + (fabs(w->v[c]) + cel) / p->dy;
            if (s > m) m = s;
        }
        w->row_a[j] = m;
    }
    double smax = 0.0;
    for (int j = 0; j < ny; ++j) if (w->row_a[j] > smax) smax = w->row_a[j];
    if (!(smax > 0.0)) return p->dt_max;
    double dt = p->cfl / smax;
    return dt < p->dt_max ? dt : p->dt_max;
}

/* S15: artificial dissipation of the level-n fields, added to level n+1.
 * nu_i = |(h_{i-1} + h_{i+1}) - 2 h_i| / ((|h_{i-1}| + |h_{i+1}|) + 2|h_i| + tiny)
 * per axis (ghost depth = adjacent interior depth); face coefficient
 * eps_{i+1/2} = max(nu_i, nu_{i+1}) on interior faces between two wet cells,
 * 0 on every other face; phi += kappa * (x term + y term). */
static void dissipation(const orc_params* p, work* w) {
    const int nx = w->nx, ny = w->ny;
    const double* h = w->h;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            double hl = h[G(i - 1, j)], hr = h[G(i + 1, j)], hb = h[G(i, j - 1)], ht = h[G(i, j + 1)];
            double hc = h[c];
            /* the two neighbours are added first so that the switch is the
             * same number seen from either side (exact mirror symmetry) */
            w->nux[c] = fabs((hl + hr) - 2.0 * hc) / ((fabs(hl) + fabs(hr)) + 2.0 * fabs(hc) + NU_TINY);
            w->nuy[c] = fabs((hb + ht) - 2.0 * hc) / ((fabs(hb) + fabs(ht)) + 2.0 * fabs(hc) + NU_TINY);
        }
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            double ee = 0.0, ew = 0.0, en = 0.0, es = 0.0;
            if (i + 1 < nx && w->wet[c] && w->wet[G(i + 1, j)]) ee = fmax(w->nux[c], w->nux[G(i + 1, j)]);
            if (i - 1 >= 0 && w->wet[c] && w->wet[G(i - 1, j)]) ew = fmax(w->nux[G(i - 1, j)], w->nux[c]);
            if (j + 1 < ny && w->wet[c] && w->wet[G(i, j + 1)]) en = fmax(w->nuy[c], w->nuy[G(i, j + 1)]);
            if (j - 1 >= 0 && w->wet[c] && w->wet[G(i, j - 1)]) es = fmax(w->nuy[G(i, j - 1)], w->nuy[c]);
            const double* fld[3] = {w->eta, w->u, w->v};
            double* out[3] = {w->e1, w->u1, w->v1};
            for (int f = 0; f < 3; ++f) {
                const double* q = fld[f];
                /* a face with zero coefficient contributes nothing, whatever the neighbour holds */
                double tx = (ee != 0.0 ? ee * (q[G(i + 1, j)] - q[c]) : 0.0)
                          - (ew != 0.0 ? ew * (q[c] - q[G(i - 1, j)]) : 0.0);
                double ty = (en != 0.0 ? en * (q[G(i, j + 1)] - q[c]) : 0.0)
                          - (es != 0.0 ? es * (q[c] - q[G(i, j - 1)]) : 0.0);
                out[f][c] = out[f][c] + p->kappa * (tx + ty);
            }
        }
}

/* S15, TVD-MacCormack form (the ablation; Davis 1984, applied to shallow
 * water by Garcia-Navarro, Alcrudo and Saviron 1992).  Per axis and per field
 * phi of level n, with the face differences D_{i+1/2} = phi_{i+1} - phi_i
 * (0 for a face outside the grid):
 *   r+_i = D_{i-1/2} D_{i+1/2} / D_{i+1/2}^2,  r-_i = D_{i-1/2} D_{i+1/2} / D_{i-1/2}^2
 *          (0 when the denominator is 0),
 *   psi(r) = max(0, min(2 r, 1)),  C(nu) = nu (1 - nu) for nu <= 1/2, else 1/4,
 *   nu_i = (|vel_i| + sqrt(g h_i)) dt / dx (0 for a dry cell), G = C(nu) (1 - psi) / 2,
 * and the face term T_{i+1/2} = (G(nu_i, r+_i) + G(nu_{i+1}, r-_{i+1})) D_{i+1/2}
 * on interior faces between two wet cells (0 on every other face);
 * phi += (T_{i+1/2} - T_{i-1/2}) + (the same along y).  In face form it
 * conserves mass; it vanishes where the differences do (lake at rest). */
static double tvd_psi(double r) { return fmax(0.0, fmin(2.0 * r, 1.0)); }
static double tvd_c(double nu) { return nu <= 0.5 ? nu * (1.0 - nu) : 0.25; }
static double tvd_ratio(double num, double den) { return den != 0.0 ? num / den : 0.0; }

/* T at the face between cells a (low side) and b (high side) along one axis:
 * dm = D below a's face, d = D of this face, dp = D above b's face. */
static double tvd_face(double dm, double d, double dp, double nua, double nub) {
    double rpa = tvd_ratio(dm * d, d * d);   /* r+ of cell a */
    double rmb = tvd_ratio(d * dp, d * d);   /* r- of cell b: D_{b-1/2} = d, D_{b+1/2} = dp */
    double ga = 0.5 * tvd_c(nua) * (1.0 - tvd_psi(rpa));
    double gb = 0.5 * tvd_c(nub) * (1.0 - tvd_psi(rmb));
    return (ga + gb) * d;
}

static void tvd_dissipation(const orc_params* p, work* w, double dt) {
    const int nx = w->nx, ny = w->ny;
    const double* h = w->h;
    const double* fld[3] = {w->eta, w->u, w->v};
    double* out[3] = {w->e1, w->u1, w->v1};
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            w->nux[c] = w->wet[c] ? (fabs(w->u[c]) + sqrt(p->g * h[c])) * dt / p->dx : 0.0;
            w->nuy[c] = w->wet[c] ? (fabs(w->v[c]) + sqrt(p->g * h[c])) * dt / p->dy : 0.0;
        }
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            for (int f = 0; f < 3; ++f) {
                const double* q = fld[f];
                /* differences of the faces i-3/2 .. i+3/2 (x) and j-3/2 .. j+3/2 (y) */
                #define DX_(ii) (((ii) >= 0 && (ii) + 1 < nx) ? q[G((ii) + 1, j)] - q[G((ii), j)] : 0.0)
                #define DY_(jj) (((jj) >= 0 && (jj) + 1 < ny) ? q[G(i, (jj) + 1)] - q[G(i, (jj))] : 0.0)
                double te = 0.0, tw = 0.0, tn = 0.0, ts = 0.0;
                if (i + 1 < nx && w->wet[c] && w->wet[G(i + 1, j)])
                    te = tvd_face(DX_(i - 1), DX_(i), DX_(i + 1), w->nux[c], w->nux[G(i + 1, j)]);
                if (i - 1 >= 0 && w->wet[c] && w->wet[G(i - 1, j)])
                    tw = tvd_face(DX_(i - 2), DX_(i - 1), DX_(i), w->nux[G(i - 1, j)], w->nux[c]);
                if (j + 1 < ny && w->wet[c] && w->wet[G(i, j + 1)])
                    tn = tvd_face(DY_(j - 1), DY_(j), DY_(j + 1), w->nuy[c], w->nuy[G(i, j + 1)]);
                if (j - 1 >= 0 && w->wet[c] && w->wet[G(i, j - 1)])
                    ts = tvd_face(DY_(j - 2), DY_(j - 1), DY_(j), w->nuy[G(i, j - 1)], w->nuy[c]);
                #undef DX_
                #undef DY_
                out[f][c] = out[f][c] + ((te - tw) + (tn - ts));
            }
        }
}

/* One full time step n -> n+1 as the 16 sub-steps, each a full-grid pass.
 * On return w->eta/u/v hold level n+1; tallies accumulate into acc[0..4]. */
static int one_step(const orc_params* p, work* w, int64_t k, double dt_in, int use_dt_in,
                    double* dt_used, double* acc) {
    const int nx = w->nx, ny = w->ny;
    int sx, sy;
    step_dirs(p->dir_cycle, k, &sx, &sy);

    depth_mask(p, w);                                              /* S1 */
    double dt = use_dt_in ? dt_in : cfl_dt(p, w);                  /* S2 */
    *dt_used = dt;
    fill_ghosts(p, w, w->eta, w->u, w->v, w->h, w->wet);           /* S3 */
    fluxes(p, w, w->h, w->u, w->v, w->qx, w->qy, w->fx, w->fy, sx, sy);       /* S4 */
    continuity(w, dt, p->dx, p->dy, w->eta, w->fx, w->fy, w->es);            /* S5 */
    friction(p, w, w->h, w->wet, w->u, w->v, w->C);                           /* S6 */
    momentum(p, w, dt, sx, sy, w->eta, w->u, w->v, w->wet, w->C,
             w->u, w->v, w->us, w->vs);                                       /* S7 */
    wetdry_fix(p, w, w->es, w->us, w->vs, w->hs, w->wets, w->row_a);          /* S8 */
    double clamp_pred = sum_rows(w->row_a, ny);
    fill_ghosts(p, w, w->es, w->us, w->vs, w->hs, w->wets);                   /* S9 */
    fluxes(p, w, w->hs, w->us, w->vs, w->qxs, w->qys, w->fxs, w->fys, -sx, -sy); /* S10 */
    continuity(w, dt, p->dx, p->dy, w->eta, w->fxs, w->fys, w->ess);          /* S11 */
    friction(p, w, w->hs, w->wets, w->us, w->vs, w->Cs);                      /* S12 */
    momentum(p, w, dt, -sx, -sy, w->es, w->us, w->vs, w->wets, w->Cs,
             w->u, w->v, w->uss, w->vss);                                     /* S13 */
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)                                              /* S14 */
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            w->e1[c] = 0.5 * (w->es[c] + w->ess[c]);
            w->u1[c] = 0.5 * (w->us[c] + w->uss[c]);
            w->v1[c] = 0.5 * (w->vs[c] + w->vss[c]);
        }
    if (p->dissipation == 1) tvd_dissipation(p, w, dt);                       /* S15 */
    else if (p->kappa != 0.0) dissipation(p, w);
    /* S16: fix of level n+1, boundary and clamp tallies, finiteness */
    wetdry_fix(p, w, w->e1, w->u1, w->v1, w->h, w->wet, w->row_b);
    double clamp_final = sum_rows(w->row_b, ny);
    acc[0] += 0.5 * clamp_pred + clamp_final;
    double bw = 0.0, be = 0.0, bs = 0.0, bn = 0.0;
    for (int j = 0; j < ny; ++j) {
        bw += 0.5 * (w->fx[FX(-1, j)] + w->fxs[FX(-1, j)]);
        be += 0.5 * (w->fx[FX(nx - 1, j)] + w->fxs[FX(nx - 1, j)]);
    }
    for (int i = 0; i < nx; ++i) {
        bs += 0.5 * (w->fy[FY(i, -1)] + w->fys[FY(i, -1)]);
        bn += 0.5 * (w->fy[FY(i, ny - 1)] + w->fys[FY(i, ny - 1)]);
    }
    acc[1] += dt * p->dy * bw;
    acc[2] -= dt * p->dy * be;
    acc[3] += dt * p->dx * bs;
    acc[4] -= dt * p->dx * bn;
    int finite = 1;
    for (int j = 0; j < ny && finite; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            if (!isfinite(w->e1[c]) || !isfinite(w->u1[c]) || !isfinite(w->v1[c])) { finite = 0; break; }
        }
    /* the new level becomes level n of the next step */
    double* t;
    t = w->eta; w->eta = w->e1; w->e1 = t;
    t = w->u; w->u = w->u1; w->u1 = t;
    t = w->v; w->v = w->v1; w->v1 = t;
    return finite ? ORC_OK : ORC_ERR_NONFINITE;
}

static int check_params(const orc_params* p) {
    if (!p || p->nx < 1 || p->ny < 1) return 0;
    if (!(p->dx > 0) || !(p->dy > 0) || !(p->g > 0) || !(p->cfl > 0)) return 0;
    if (!(p->h_dry > 0) || !(p->dt_max > 0) || !(p->kappa >= 0) || !(p->manning_n >= 0)) return 0;
    for (int s = 0; s < 4; ++s) if (p->bc[s] < BC_WALL || p->bc[s] > BC_OUTFLOW) return 0;
    if (p->dir_cycle < 0 || p->dir_cycle > 7) return 0;
    if (p->friction < 0 || p->friction > 1 || p->dissipation < 0 || p->dissipation > 1) return 0;
    return 1;
}

static void load(const orc_params* p, work* w, const double* z, const double* nfield,
                 const double* eta, const double* u, const double* v) {
    const int nx = w->nx, ny = w->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j), k = (size_t)j * nx + i;
            w->z[c] = z[k];
            double n = nfield ? nfield[k] : p->manning_n;
            w->n2[c] = n * n;
            w->eta[c] = eta[k]; w->u[c] = u[k]; w->v[c] = v[k];
        }
    /* ghost bed = adjacent interior bed */
    for (int j = 0; j < ny; ++j) { w->z[G(-1, j)] = w->z[G(0, j)]; w->z[G(nx, j)] = w->z[G(nx - 1, j)]; }
    for (int i = 0; i < nx; ++i) { w->z[G(i, -1)] = w->z[G(i, 0)]; w->z[G(i, ny)] = w->z[G(i, ny - 1)]; }
}

/* ------------------------------------------------------------------ */
/* Public entry points (called from Python through ctypes)             */
/* ------------------------------------------------------------------ */

/* Advance eta/u/v (in place) by nsteps steps starting at step index step0.
 * dt_fixed (nullable, nsteps values) replaces S2; dt_out (nullable) receives
 * the step sizes used; acc[5] accumulates clamp volume and the boundary
 * inflow volumes of sides W, E, S, N (m^3).  Returns 0, 1 (bad argument) or
 * 3 (a non-finite value appeared; the state is that of the failing step). */
int orc_run(const orc_params* p, const double* z, const double* nfield,
            double* eta, double* u, double* v, int64_t step0, int32_t nsteps,
            const double* dt_fixed, double* dt_out, double* acc, int32_t nthreads) {
    if (!check_params(p) || !z || !eta || !u || !v || !acc || nsteps < 0) return ORC_ERR_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    work wk, *w = &wk;
    if (!work_alloc(w, p->nx, p->ny)) return ORC_ERR_ARG;
    load(p, w, z, nfield, eta, u, v);
    int st = ORC_OK;
    for (int32_t s = 0; s < nsteps; ++s) {
        double dt;
        st = one_step(p, w, step0 + s, dt_fixed ? dt_fixed[s] : 0.0, dt_fixed != NULL, &dt, acc);
        if (dt_out) dt_out[s] = dt;
        if (st != ORC_OK) break;
    }
    for (int j = 0; j < p->ny; ++j)
        for (int i = 0; i < p->nx; ++i) {
            size_t c = G(i, j), k = (size_t)j * p->nx + i;
            eta[k] = w->eta[c]; u[k] = w->u[c]; v[k] = w->v[c];
        }
    work_free(w);
    return st;
}

/* S2 alone on a given state. */
double orc_dt(const orc_params* p, const double* z, const double* eta, const double* u,
              const double* v) {
    if (!check_params(p)) return -1.0;
    work wk, *w = &wk;
    if (!work_alloc(w, p->nx, p->ny)) return -1.0;
    load(p, w, z, NULL, eta, u, v);
    depth_mask(p, w);
    double dt = cfl_dt(p, w);
    work_free(w);
    return dt;
}

/* Volume sum(h) dx dy, plain sequential sum (rows in order, i fastest). */
double orc_volume(const orc_params* p, const double* z, const double* eta) {
    double s = 0.0;
    size_t n = (size_t)p->nx * (size_t)p->ny;
    for (size_t k = 0; k < n; ++k) s += eta[k] - z[k];
    return s * p->dx * p->dy;
}

/* Set-state normalisation: a depth below -1e-12 m is rejected (returns 1);
 * a smaller negative depth is clamped (eta = z); dry cells (h <= h_dry)
 * get zero velocity. */
int orc_prepare_state(const orc_params* p, const double* z, double* eta, double* u, double* v) {
    if (!check_params(p)) return ORC_ERR_ARG;
    size_t n = (size_t)p->nx * (size_t)p->ny;
    for (size_t k = 0; k < n; ++k) {
        if (!isfinite(eta[k]) || !isfinite(u[k]) || !isfinite(v[k]) || !isfinite(z[k])) return ORC_ERR_ARG;
        if (eta[k] - z[k] < -1e-12) return ORC_ERR_ARG;
    }
    for (size_t k = 0; k < n; ++k) {
        double d = eta[k] - z[k];
        if (d < 0.0) { eta[k] = z[k]; d = 0.0; }
        if (d <= p->h_dry) { u[k] = 0.0; v[k] = 0.0; }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Discrete adjoint (reverse mode) of the step, for gradient checks    */
/* ------------------------------------------------------------------ */
/* Scope: dt frozen per step (the CFL minimum is not differentiated),
 * kappa = 0 (S15 off) and a fully wet domain in every stage (S8/S16 are then
 * the identity); orc_adjoint returns 5 otherwise.  Each forward sub-step
 * below has its reverse: given the cotangent of its outputs it adds the
 * cotangents of its inputs, over the same full-grid arrays. */
enum { ORC_ERR_NOT_WET = 5 };

typedef struct {
    double *le, *lu, *lv, *lh;        /* level n (with ghosts) */
    double *lC, *lfx, *lfy, *lqx, *lqy;
    double *les, *lus, *lvs, *lhs;    /* predicted (with ghosts) */
    double *lCs, *lfxs, *lfys, *lqxs, *lqys;
    double *ln2;                      /* per cell */
    double *lz;                       /* per cell: cotangent of the bed z of this step */
} adjw;

static void adjw_free(adjw* a) {
    void* ptrs[] = {a->le, a->lu, a->lv, a->lh, a->lC, a->lfx, a->lfy, a->lqx, a->lqy, a->les, a->lus,
                    a->lvs, a->lhs, a->lCs, a->lfxs, a->lfys, a->lqxs, a->lqys, a->ln2, a->lz};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    memset(a, 0, sizeof(*a));
}

static int adjw_alloc(adjw* a, int nx, int ny) {
    memset(a, 0, sizeof(*a));
    size_t nc = (size_t)(nx + 2) * (size_t)(ny + 2);
    size_t nfx = (size_t)(nx + 1) * (size_t)ny, nfy = (size_t)nx * (size_t)(ny + 1);
    double** cells[] = {&a->le, &a->lu, &a->lv, &a->lh, &a->lC, &a->lqx, &a->lqy, &a->les, &a->lus,
                        &a->lvs, &a->lhs, &a->lCs, &a->lqxs, &a->lqys, &a->ln2, &a->lz};
    for (size_t k = 0; k < sizeof(cells) / sizeof(cells[0]); ++k)
        if (!(*cells[k] = calloc(nc, sizeof(double)))) { adjw_free(a); return 0; }
    if (!(a->lfx = calloc(nfx, sizeof(double))) || !(a->lfy = calloc(nfy, sizeof(double))) ||
        !(a->lfxs = calloc(nfx, sizeof(double))) || !(a->lfys = calloc(nfy, sizeof(double)))) {
        adjw_free(a);
        return 0;
    }
    return 1;
}

static void adjw_zero(adjw* a, int nx, int ny) {
    size_t nc = (size_t)(nx + 2) * (size_t)(ny + 2);
    size_t nfx = (size_t)(nx + 1) * (size_t)ny, nfy = (size_t)nx * (size_t)(ny + 1);
    double* cells[] = {a->le, a->lu, a->lv, a->lh, a->lC, a->lqx, a->lqy, a->les, a->lus, a->lvs, a->lhs,
                       a->lCs, a->lqxs, a->lqys};
    for (size_t k = 0; k < sizeof(cells) / sizeof(cells[0]); ++k) memset(cells[k], 0, nc * sizeof(double));
    memset(a->lfx, 0, nfx * sizeof(double)); memset(a->lfy, 0, nfy * sizeof(double));
    memset(a->lfxs, 0, nfx * sizeof(double)); memset(a->lfys, 0, nfy * sizeof(double));
}

/* reverse of fill_ghosts: fold the ghost cotangents into the adjacent cells */
static void adj_ghosts(const orc_params* p, work* w, const double* h, double* le, double* lu, double* lv,
                       double* lh) {
    const int nx = w->nx, ny = w->ny;
    for (int j = 0; j < ny; ++j)
        for (int side = SIDE_W; side <= SIDE_E; ++side) {
            int ii = (side == SIDE_W) ? 0 : nx - 1, ig = (side == SIDE_W) ? -1 : nx;
            double sgn = (side == SIDE_W) ? 1.0 : -1.0;
            size_t a = G(ii, j), b = G(ig, j);
            le[a] += le[b]; lh[a] += lh[b];
            switch (p->bc[side]) {
            case BC_WALL: lu[a] -= lu[b]; lv[a] += lv[b]; break;
            case BC_INFLOW:
                if (h[a] > p->h_dry) lh[a] += -sgn * p->q_in[side] / (h[a] * h[a]) * lu[b];
                break;
            default: lu[a] += lu[b]; lv[a] += lv[b]; break;
            }
            le[b] = lh[b] = lu[b] = lv[b] = 0.0;
        }
    for (int i = 0; i < nx; ++i)
        for (int side = SIDE_S; side <= SIDE_N; ++side) {
            int jj = (side == SIDE_S) ? 0 : ny - 1, jg = (side == SIDE_S) ? -1 : ny;
            double sgn = (side == SIDE_S) ? 1.0 : -1.0;
            size_t a = G(i, jj), b = G(i, jg);
            le[a] += le[b]; lh[a] += lh[b];
            switch (p->bc[side]) {
            case BC_WALL: lv[a] -= lv[b]; lu[a] += lu[b]; break;
            case BC_INFLOW:
                if (h[a] > p->h_dry) lh[a] += -sgn * p->q_in[side] / (h[a] * h[a]) * lv[b];
                break;
            default: lu[a] += lu[b]; lv[a] += lv[b]; break;
            }
            le[b] = lh[b] = lu[b] = lv[b] = 0.0;
        }
}

/* reverse of fluxes(): face cotangents to the cell fluxes, then to h, u, v */
static void adj_fluxes(const orc_params* p, work* w, const double* h, const double* u, const double* v,
                       const double* lfx, const double* lfy, double* lqx, double* lqy, double* lh, double* lu,
                       double* lv, int sx, int sy) {
    const int nx = w->nx, ny = w->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = -1; i < nx; ++i) {
            double l = lfx[FX(i, j)];
            if (i == -1 || i == nx - 1) {
                int side = (i == -1) ? SIDE_W : SIDE_E, inner = (i == -1) ? 0 : nx - 1;
                if (p->bc[side] == BC_OUTFLOW) lqx[G(inner, j)] += l;
            } else {
                lqx[(sx > 0) ? G(i + 1, j) : G(i, j)] += l;
            }
        }
    for (int j = -1; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double l = lfy[FY(i, j)];
            if (j == -1 || j == ny - 1) {
                int side = (j == -1) ? SIDE_S : SIDE_N, inner = (j == -1) ? 0 : ny - 1;
                if (p->bc[side] == BC_OUTFLOW) lqy[G(i, inner)] += l;
            } else {
                lqy[(sy > 0) ? G(i, j + 1) : G(i, j)] += l;
            }
        }
    for (int j = -1; j <= ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            int gi = (i < 0 || i >= nx), gj = (j < 0 || j >= ny);
            if (gi && gj) continue;
            size_t c = G(i, j);
            lh[c] += u[c] * lqx[c] + v[c] * lqy[c];
            lu[c] += h[c] * lqx[c];
            lv[c] += h[c] * lqy[c];
        }
}

/* reverse of continuity() */
static void adj_continuity(work* w, double dt, double dx, double dy, const double* lout, double* leta_n,
                           double* lfx, double* lfy) {
    const int nx = w->nx, ny = w->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double l = lout[G(i, j)];
            leta_n[G(i, j)] += l;
            lfx[FX(i, j)] -= dt / dx * l;
            lfx[FX(i - 1, j)] += dt / dx * l;
            lfy[FY(i, j)] -= dt / dy * l;
            lfy[FY(i, j - 1)] += dt / dy * l;
        }
}

/* reverse of friction(): C = g n2 |U| / h^(4/3) on wet cells */
static void adj_friction(const orc_params* p, work* w, const double* h, const unsigned char* wet,
                         const double* u, const double* v, const double* C, const double* lC, double* lh,
                         double* lu, double* lv, double* ln2) {
    const int nx = w->nx, ny = w->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            if (!wet[c]) continue;
            double mag = sqrt(u[c] * u[c] + v[c] * v[c]);
            double P = pow(h[c], 4.0 / 3.0);
            double l = lC[c];
            ln2[c] += p->g * mag / P * l;
            if (mag > 0.0) {
                lu[c] += p->g * w->n2[c] * (u[c] / mag) / P * l;
                lv[c] += p->g * w->n2[c] * (v[c] / mag) / P * l;
            }
            lh[c] += -(4.0 / 3.0) * C[c] / h[c] * l;
        }
}

/* reverse of momentum() */
static void adj_momentum(const orc_params* p, work* w, double dt, int sx, int sy, const double* eta,
                         const double* u, const double* v, const unsigned char* wet, const double* C,
                         const double* u_out, const double* v_out, const double* lu_out, const double* lv_out,
                         double* leta, double* lu, double* lv, double* lC, double* lu_n, double* lv_n) {
    const int nx = w->nx, ny = w->ny;
    const double* z = w->z;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            size_t xn = (sx > 0) ? G(i + 1, j) : G(i - 1, j);
            size_t yn = (sy > 0) ? G(i, j + 1) : G(i, j - 1);
            int xwall = (!wet[xn] && z[xn] > eta[c]), ywall = (!wet[yn] && z[yn] > eta[c]);
            double ex = xwall ? eta[c] : eta[xn], ey = ywall ? eta[c] : eta[yn];
            (void)ex; (void)ey;
            double dux = sx * (u[xn] - u[c]), dvx = sx * (v[xn] - v[c]);
            double duy = sy * (u[yn] - u[c]), dvy = sy * (v[yn] - v[c]);
            double den = 1.0 + dt * C[c];
            double lo_u = lu_out[c], lo_v = lv_out[c];
            lu_n[c] += lo_u / den;
            lv_n[c] += lo_v / den;
            double lAu = -dt * lo_u / den, lAv = -dt * lo_v / den;
            double lden = -(u_out[c] * lo_u + v_out[c] * lo_v) / den;
            lC[c] += dt * lden;
            double ldux = u[c] / p->dx * lAu, lduy = v[c] / p->dy * lAu, ldex = p->g / p->dx * lAu;
            double ldvx = u[c] / p->dx * lAv, ldvy = v[c] / p->dy * lAv, ldey = p->g / p->dy * lAv;
            lu[c] += dux / p->dx * lAu + dvx / p->dx * lAv;
            lv[c] += duy / p->dy * lAu + dvy / p->dy * lAv;
            lu[xn] += sx * ldux; lu[c] -= sx * ldux;
            lv[xn] += sx * ldvx; lv[c] -= sx * ldvx;
            lu[yn] += sy * lduy; lu[c] -= sy * lduy;
            lv[yn] += sy * ldvy; lv[c] -= sy * ldvy;
            double lex = sx * ldex, ley = sy * ldey;
            leta[c] -= sx * ldex + sy * ldey;
            if (xwall) leta[c] += lex; else leta[xn] += lex;
            if (ywall) leta[c] += ley; else leta[yn] += ley;
        }
}

static int all_wet(work* w, const unsigned char* wet) {
    for (int j = 0; j < w->ny; ++j)
        for (int i = 0; i < w->nx; ++i)
            if (!wet[G(i, j)]) return 0;
    return 1;
}

/* Forward sub-steps S1-S14 of step k from the current w->eta/u/v, keeping
 * every intermediate in w; the new level is in w->e1/u1/v1 (S15 off, S16 the
 * identity when fully wet).  Returns 0, or ORC_ERR_NOT_WET. */
static int fwd_keep(const orc_params* p, work* w, int64_t k, double dt, int* sx, int* sy) {
    const int ny = w->ny;
    step_dirs(p->dir_cycle, k, sx, sy);
    depth_mask(p, w);
    if (!all_wet(w, w->wet)) return ORC_ERR_NOT_WET;
    fill_ghosts(p, w, w->eta, w->u, w->v, w->h, w->wet);
    fluxes(p, w, w->h, w->u, w->v, w->qx, w->qy, w->fx, w->fy, *sx, *sy);
    continuity(w, dt, p->dx, p->dy, w->eta, w->fx, w->fy, w->es);
    friction(p, w, w->h, w->wet, w->u, w->v, w->C);
    momentum(p, w, dt, *sx, *sy, w->eta, w->u, w->v, w->wet, w->C, w->u, w->v, w->us, w->vs);
    wetdry_fix(p, w, w->es, w->us, w->vs, w->hs, w->wets, w->row_a);
    if (sum_rows(w->row_a, ny) != 0.0 || !all_wet(w, w->wets)) return ORC_ERR_NOT_WET;
    fill_ghosts(p, w, w->es, w->us, w->vs, w->hs, w->wets);
    fluxes(p, w, w->hs, w->us, w->vs, w->qxs, w->qys, w->fxs, w->fys, -*sx, -*sy);
    continuity(w, dt, p->dx, p->dy, w->eta, w->fxs, w->fys, w->ess);
    friction(p, w, w->hs, w->wets, w->us, w->vs, w->Cs);
    momentum(p, w, dt, -*sx, -*sy, w->es, w->us, w->vs, w->wets, w->Cs, w->u, w->v, w->uss, w->vss);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < w->nx; ++i) {
            size_t c = G(i, j);
            w->e1[c] = 0.5 * (w->es[c] + w->ess[c]);
            w->u1[c] = 0.5 * (w->us[c] + w->uss[c]);
            w->v1[c] = 0.5 * (w->vs[c] + w->vss[c]);
            if (!(w->e1[c] - w->z[c] > p->h_dry)) return ORC_ERR_NOT_WET;
        }
    return ORC_OK;
}

/* Reverse of one step: given the cotangent (le1, lu1, lv1) of level n+1 in
 * the interior of a->le/lu/lv... the caller passes them in lin_*; on return
 * a->le/lu/lv hold the cotangent of level n and a->ln2 has accumulated the
 * cotangent of n^2 (per cell). */
static void adj_step(const orc_params* p, work* w, adjw* a, double dt, int sx, int sy, const double* le1,
                     const double* lu1, const double* lv1) {
    const int nx = w->nx, ny = w->ny;
    double* ln2 = a->ln2;
    adjw_zero(a, nx, ny);
    /* S14: average; the predicted state receives half directly */
    double *less = calloc((size_t)(nx + 2) * (ny + 2), sizeof(double));
    double *luss = calloc((size_t)(nx + 2) * (ny + 2), sizeof(double));
    double *lvss = calloc((size_t)(nx + 2) * (ny + 2), sizeof(double));
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = G(i, j);
            size_t k = (size_t)j * nx + i;
            a->les[c] += 0.5 * le1[k]; less[c] = 0.5 * le1[k];
            a->lus[c] += 0.5 * lu1[k]; luss[c] = 0.5 * lu1[k];
            a->lvs[c] += 0.5 * lv1[k]; lvss[c] = 0.5 * lv1[k];
        }
    /* S13: corrector momentum (differenced state: predicted; base: level n) */
    adj_momentum(p, w, dt, -sx, -sy, w->es, w->us, w->vs, w->wets, w->Cs, w->uss, w->vss, luss, lvss,
                 a->les, a->lus, a->lvs, a->lCs, a->lu, a->lv);
    /* S12: corrector friction */
    adj_friction(p, w, w->hs, w->wets, w->us, w->vs, w->Cs, a->lCs, a->lhs, a->lus, a->lvs, ln2);
    /* S11: corrector continuity */
    adj_continuity(w, dt, p->dx, p->dy, less, a->le, a->lfxs, a->lfys);
    /* S10: corrector fluxes */
    adj_fluxes(p, w, w->hs, w->us, w->vs, a->lfxs, a->lfys, a->lqxs, a->lqys, a->lhs, a->lus, a->lvs, -sx, -sy);
    /* S9: ghosts of the predicted state */
    adj_ghosts(p, w, w->hs, a->les, a->lus, a->lvs, a->lhs);
    /* S8: the fix is the identity (wet, no clamp); h* = eta* - z */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) { size_t c = G(i, j); a->les[c] += a->lhs[c]; a->lz[c] -= a->lhs[c]; }
    /* S7: predictor momentum (differenced and base state: level n) */
    adj_momentum(p, w, dt, sx, sy, w->eta, w->u, w->v, w->wet, w->C, w->us, w->vs, a->lus, a->lvs,
                 a->le, a->lu, a->lv, a->lC, a->lu, a->lv);
    /* S6: predictor friction */
    adj_friction(p, w, w->h, w->wet, w->u, w->v, w->C, a->lC, a->lh, a->lu, a->lv, ln2);
    /* S5: predictor continuity */
    adj_continuity(w, dt, p->dx, p->dy, a->les, a->le, a->lfx, a->lfy);
    /* S4: predictor fluxes */
    adj_fluxes(p, w, w->h, w->u, w->v, a->lfx, a->lfy, a->lqx, a->lqy, a->lh, a->lu, a->lv, sx, sy);
    /* S3: ghosts of level n */
    adj_ghosts(p, w, w->h, a->le, a->lu, a->lv, a->lh);
    /* S1: h = eta - z */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) { size_t c = G(i, j); a->le[c] += a->lh[c]; a->lz[c] -= a->lh[c]; }
    free(less); free(luss); free(lvss);
}

/* Gradient of L = 1/2 sum_{k=1..T} sum_g (eta_g^k - obs[k-1][g])^2 with
 * respect to the per-cell Manning n field, the bed elevation z (which enters
 * every stage through the depth h = eta - z, and the ghost cells through
 * their copy of the adjacent bed) and the initial eta (and u, v), by the
 * discrete adjoint of T steps from step index step0 with the given frozen
 * step sizes.  Returns 0, 1 (bad argument), 3 (non-finite) or 5 (a stage was
 * not fully wet, or kappa != 0). */
int orc_adjoint(const orc_params* p, const double* z, const double* nfield, const double* eta0,
                const double* u0, const double* v0, int64_t step0, int32_t T, const double* dt,
                const int64_t* gauges, int32_t ng, const double* obs, double* loss, double* grad_n,
                double* grad_eta0, double* grad_u0, double* grad_v0, double* grad_z) {
    if (!check_params(p) || !z || !nfield || !eta0 || !u0 || !v0 || !dt || T < 0 || ng < 0 || !loss) return ORC_ERR_ARG;
    if (p->kappa != 0.0 || p->friction != 0 || p->dissipation != 0) return ORC_ERR_NOT_WET;
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny, nc = (size_t)(nx + 2) * (ny + 2);
    for (int32_t g = 0; g < ng; ++g)
        if (gauges[g] < 0 || (size_t)gauges[g] >= n) return ORC_ERR_ARG;
    work wk, *w = &wk;
    if (!work_alloc(w, nx, ny)) return ORC_ERR_ARG;
    adjw aw, *a = &aw;
    if (!adjw_alloc(a, nx, ny)) { work_free(w); return ORC_ERR_ARG; }
    /* forward, keeping every level (interior, dense) */
    double* st = malloc((size_t)(T + 1) * 3 * n * sizeof(double));
    double *le1 = malloc(n * sizeof(double)), *lu1 = malloc(n * sizeof(double)), *lv1 = malloc(n * sizeof(double));
    double* gn = calloc(nc, sizeof(double));
    double* gz = calloc(nc, sizeof(double));
    if (!st || !le1 || !lu1 || !lv1 || !gn || !gz) { free(st); free(le1); free(lu1); free(lv1); free(gn); free(gz); adjw_free(a); work_free(w); return ORC_ERR_ARG; }
    load(p, w, z, nfield, eta0, u0, v0);
    int rc = ORC_OK;
    double L = 0.0;
    for (int32_t s = 0; s <= T && rc == ORC_OK; ++s) {
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = G(i, j), k = (size_t)j * nx + i;
                st[(size_t)s * 3 * n + k] = w->eta[c];
                st[(size_t)s * 3 * n + n + k] = w->u[c];
                st[(size_t)s * 3 * n + 2 * n + k] = w->v[c];
            }
        if (s >= 1)
            for (int32_t g = 0; g < ng; ++g) {
                double r = st[(size_t)s * 3 * n + gauges[g]] - obs[(size_t)(s - 1) * ng + g];
                L += 0.5 * r * r;
            }
        if (s == T) break;
        int sx, sy;
        rc = fwd_keep(p, w, step0 + s, dt[s], &sx, &sy);
        double* t;
        t = w->eta; w->eta = w->e1; w->e1 = t;
        t = w->u; w->u = w->u1; w->u1 = t;
        t = w->v; w->v = w->v1; w->v1 = t;
    }
    if (rc == ORC_OK && !isfinite(L)) rc = ORC_ERR_NONFINITE;
    if (rc == ORC_OK) {
        *loss = L;
        /* cotangent of level T: the gauge residuals */
        memset(le1, 0, n * sizeof(double)); memset(lu1, 0, n * sizeof(double)); memset(lv1, 0, n * sizeof(double));
        if (T >= 1)
            for (int32_t g = 0; g < ng; ++g)
                le1[gauges[g]] += st[(size_t)T * 3 * n + gauges[g]] - obs[(size_t)(T - 1) * ng + g];
        for (int32_t s = T - 1; s >= 0; --s) {
            /* recompute step s from level s, then reverse it */
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t c = G(i, j), k = (size_t)j * nx + i;
                    w->eta[c] = st[(size_t)s * 3 * n + k];
                    w->u[c] = st[(size_t)s * 3 * n + n + k];
                    w->v[c] = st[(size_t)s * 3 * n + 2 * n + k];
                }
            int sx, sy;
            fwd_keep(p, w, step0 + s, dt[s], &sx, &sy);
            memset(a->ln2, 0, nc * sizeof(double));
            memset(a->lz, 0, nc * sizeof(double));
            adj_step(p, w, a, dt[s], sx, sy, le1, lu1, lv1);
            for (size_t c = 0; c < nc; ++c) { gn[c] += a->ln2[c]; gz[c] += a->lz[c]; }
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t c = G(i, j), k = (size_t)j * nx + i;
                    le1[k] = a->le[c]; lu1[k] = a->lu[c]; lv1[k] = a->lv[c];
                }
            if (s >= 1)
                for (int32_t g = 0; g < ng; ++g)
                    le1[gauges[g]] += st[(size_t)s * 3 * n + gauges[g]] - obs[(size_t)(s - 1) * ng + g];
        }
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = G(i, j), k = (size_t)j * nx + i;
                if (grad_n) grad_n[k] = gn[c] * 2.0 * nfield[k];  /* d(n^2)/dn */
                if (grad_eta0) grad_eta0[k] = le1[k];
                if (grad_u0) grad_u0[k] = lu1[k];
                if (grad_v0) grad_v0[k] = lv1[k];
                if (grad_z) grad_z[k] = gz[c];
            }
    }
    free(st); free(le1); free(lu1); free(lv1); free(gn); free(gz);
    adjw_free(a);
    work_free(w);
    return rc;
}
