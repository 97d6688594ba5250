/*
 * maclab_oracle.c -- plain FP64 CPU oracle of the MacLAB time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct reference the
 * CUDA library is checked against.  Only the tests, the smoke check and the
 * CPU-baseline / reference legs of the benchmark build, load or call it; the
 * product path never does, and it shares no code, table or header with the
 * CUDA library.
 *
 * What it computes (Zhou, "Macroscopic Lattice Boltzmann Method"):
 *   Eq. (2)  f_a^eq = w_a rho (1 + 3 e_ai u_i/e^2 + 9/2 e_ai e_aj u_i u_j/e^4
 *                              - 3/2 u_i u_i/e^2)
 *   Eq. (4)  rho(x, t)  = sum_a f_a^eq(x - e_a dt, t - dt)
 *   Eq. (5)  u_i(x, t)  = 1/rho(x, t) sum_a e_ai f_a^eq(x - e_a dt, t - dt)
 *            (the printed e_aj is read as e_ai, as in Eq. (12) of Methods)
 *   procedure (i)-(v) after Eq. (6): equilibria from (rho, u), update by
 *   Eqs. (4)-(5), then the boundary conditions, repeat.
 *
 * Units.  e_a = e c_a with c_a in {-1,0,1}^d, so the upstream point
 * x - e_a dt (dt = dx/e) is the lattice node x - c_a.  Velocities are held in
 * lattice units ut = u/e, so e_ai u_i / e^2 = c_a . ut and Eq. (2) becomes
 *     f_a^eq = w_a rho (1 + 3 c.ut + 4.5 (c.ut)^2 - 1.5 ut.ut).
 * Everything here works in those units with rho itself (not rho - 1).
 *
 * Boundaries.  Wall nodes keep their (rho, u): the paper retains physical
 * variables on walls with no calculation there (Tests 2, 3 and 5).  They still
 * act as upstream sources for fluid neighbours.  Periodic axes wrap (Tests 1
 * and 4).  A fluid node whose upstream node would leave a non-periodic axis is
 * an input error (returned, never clamped).
 *
 * Body force (Test 2).  After the division of Eq. (5) the lattice velocity
 * gains force[i] (the pressure-gradient term of Test 2 in lattice units; its
 * sign is taken so that the closed form Eq. (8) holds).
 *
 * Threads.  With OpenMP the node loops run on several host threads.  Every
 * output value is still formed by one thread with exactly the operations and
 * operand order of the single-thread loop, so results are bitwise independent
 * of the thread count (oracle_set_threads); no sum is split across threads.
 *
 * Build: plain C99, -O2 -ffp-contract=off, no -ffast-math, -fopenmp if the
 * compiler has it (without it every loop runs on one thread).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads for the node loops (OpenMP builds); returns the count in use. */
int oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* D2Q9 velocities in the order listed after Eq. (1), alpha = 0..8. */
static const int D2Q9_C[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
/* D2Q9 weights given after Eq. (2): 4/9, 1/9 (alpha 1-4), 1/36 (alpha 5-8). */
static const double D2Q9_W[9] = {
    4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* D3Q19 velocities in the order listed with the five simulations. */
static const int D3Q19_C[19][3] = {
    {0, 0, 0},   {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},   {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {-1, 1, 0},
    {1, -1, 0},  {0, 1, 1},  {0, -1, -1}, {0, -1, 1}, {0, 1, -1},
    {1, 0, 1},   {-1, 0, -1}, {-1, 0, 1}, {1, 0, -1}};
/* D3Q19 weights: 1/3 (alpha 0), 1/18 (alpha 1-6), 1/36 (alpha 7-18). */
static const double D3Q19_W[19] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

enum { ORACLE_OK = 0, ORACLE_BAD_ARG = -1, ORACLE_OUTSIDE = -2, ORACLE_NOMEM = -3 };

typedef struct {
    int d, q;
    const int (*c)[3];
    const double *w;
} lattice_t;

static int get_lattice(int lattice, lattice_t *L) {
    if (lattice == 0) { L->d = 2; L->q = 9; L->c = D2Q9_C; L->w = D2Q9_W; return 0; }
    if (lattice == 1) { L->d = 3; L->q = 19; L->c = D3Q19_C; L->w = D3Q19_W; return 0; }
    return -1;
}

/* Lattice tables, exported so the tests can check them against the paper. */
int oracle_lattice_table(int lattice, int *c_out, double *w_out) {
    lattice_t L;
    if (get_lattice(lattice, &L)) return ORACLE_BAD_ARG;
    for (int a = 0; a < L.q; ++a) {
        for (int i = 0; i < 3; ++i) c_out[3 * a + i] = L.c[a][i];
        w_out[a] = L.w[a];
    }
    return L.q;
}

/* Eq. (2) in lattice units: f_a^eq(rho, ut) for direction a. */
static double feq(const lattice_t *L, int a, double rho, const double *ut) {
    double cu = 0.0, uu = 0.0;
    for (int i = 0; i < L->d; ++i) {
        cu += (double)L->c[a][i] * ut[i];
        uu += ut[i] * ut[i];
    }
    return L->w[a] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

double oracle_feq(int lattice, int a, double rho, const double *ut) {
    lattice_t L;
    if (get_lattice(lattice, &L) || a < 0 || a >= L.q) return 0.0;
    return feq(&L, a, rho, ut);
}

/* Upstream coordinate x - c along one axis; -1 if it leaves a closed axis. */
static int64_t upstream(int64_t x, int c, int64_t n, int periodic) {
    int64_t y = x - c;
    if (y < 0 || y >= n) {
        if (!periodic) return -1;
        y = (y % n + n) % n;
    }
    return y;
}

/*
 * One MacLAB step.  rho/u: N values and d*N values (component-major SoA,
 * u[i*N + node], node = (z*ny + y)*nx + x).  wall: N bytes, nonzero = wall
 * node, or NULL.  force: d lattice-unit increments added after Eq. (5).
 */
int oracle_step(int lattice, int64_t nx, int64_t ny, int64_t nz, uint32_t periodic,
                const uint8_t *wall, const double *rho, const double *u,
                const double *force, double *rho_out, double *u_out) {
    lattice_t L;
    if (get_lattice(lattice, &L)) return ORACLE_BAD_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || (L.d == 2 && nz != 1)) return ORACLE_BAD_ARG;
    const int64_t n[3] = {nx, ny, nz};
    const int64_t N = nx * ny * nz;
    int outside = 0;  /* set when a fluid node's upstream node leaves a closed axis */
#pragma omp parallel for schedule(static)
    for (int64_t node = 0; node < N; ++node) {
        const int64_t x[3] = {node % nx, (node / nx) % ny, node / (nx * ny)};
        if (wall && wall[node]) {
            /* step (iv): physical variables retained on the wall */
            rho_out[node] = rho[node];
            for (int i = 0; i < L.d; ++i) u_out[i * N + node] = u[i * N + node];
            continue;
        }
        double rho_new = 0.0, mom[3] = {0.0, 0.0, 0.0};
        int bad = 0;
        for (int a = 0; a < L.q && !bad; ++a) {
            int64_t y[3] = {0, 0, 0};
            for (int i = 0; i < 3; ++i) {
                y[i] = upstream(x[i], L.c[a][i], n[i], (periodic >> i) & 1u);
                if (y[i] < 0) bad = 1;
            }
            if (bad) break;
            const int64_t src = (y[2] * ny + y[1]) * nx + y[0];
            double ut[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < L.d; ++i) ut[i] = u[i * N + src];
            const double f = feq(&L, a, rho[src], ut);
            rho_new += f;                                       /* Eq. (4) */
            for (int i = 0; i < L.d; ++i) mom[i] += (double)L.c[a][i] * f;  /* Eq. (5) */
        }
        if (bad) {
#pragma omp atomic write
            outside = 1;
            continue;
        }
        rho_out[node] = rho_new;
        for (int i = 0; i < L.d; ++i)
            u_out[i * N + node] = mom[i] / rho_new + (force ? force[i] : 0.0);
    }
    return outside ? ORACLE_OUTSIDE : ORACLE_OK;
}

/* Step (v): repeat the update nsteps times (ping-pong). In-place on rho/u. */
int oracle_run(int lattice, int64_t nx, int64_t ny, int64_t nz, uint32_t periodic,
               const uint8_t *wall, double *rho, double *u, const double *force,
               int64_t nsteps) {
    lattice_t L;
    if (get_lattice(lattice, &L)) return ORACLE_BAD_ARG;
    const int64_t N = nx * ny * nz;
    double *r2 = (double *)malloc(sizeof(double) * (size_t)N);
    double *u2 = (double *)malloc(sizeof(double) * (size_t)N * (size_t)L.d);
    if (!r2 || !u2) { free(r2); free(u2); return ORACLE_NOMEM; }
    double *ra = rho, *ua = u, *rb = r2, *ub = u2;
    int rc = ORACLE_OK;
    for (int64_t s = 0; s < nsteps && rc == ORACLE_OK; ++s) {
        rc = oracle_step(lattice, nx, ny, nz, periodic, wall, ra, ua, force, rb, ub);
        double *t = ra; ra = rb; rb = t;
        t = ua; ua = ub; ub = t;
    }
    if (ra != rho) {
        memcpy(rho, ra, sizeof(double) * (size_t)N);
        memcpy(u, ua, sizeof(double) * (size_t)N * (size_t)L.d);
    }
    free(r2);
    free(u2);
    return rc;
}

/*
 * Adjoint (reverse-mode derivative) of oracle_step.  Not in the paper; it is
 * the chain rule applied to Eqs. (2), (4), (5) and the force term, written out
 * plainly.  Inputs: the state (rho, u) that oracle_step consumed, the adjoints
 * lam_rho_next / lam_u_next of its outputs.  Outputs: lam_rho / lam_u, the
 * adjoints of its inputs, and grad_force[i] += sum over fluid nodes of
 * lam_u_next[i] (d output / d force = identity on fluid nodes).
 *
 * For a fluid node x with outputs rho' = sum_a F_a and ut' = m/rho' + force,
 * m = sum_a c_a F_a, F_a = f_a^eq(rho(x - c_a), ut(x - c_a)):
 *   dL/drho' (through both outputs) = lam_rho'(x) - sum_i lam_u'_i m_i / rho'^2
 *   dL/dm_i                         = lam_u'_i / rho'
 * and each F_a then passes g_a = dL/drho' + c_a . dL/dm back to its source y
 * through dF_a/drho = w_a (1 + 3 c.ut + 4.5 (c.ut)^2 - 1.5 ut.ut) and
 * dF_a/dut = w_a rho (3 c + 9 (c.ut) c - 3 ut).  A wall node's output equals
 * its input, so its incoming adjoint passes straight through.
 */
int oracle_adjoint_step(int lattice, int64_t nx, int64_t ny, int64_t nz, uint32_t periodic,
                        const uint8_t *wall, const double *rho, const double *u,
                        const double *force, const double *lam_rho_next,
                        const double *lam_u_next, double *lam_rho, double *lam_u,
                        double *grad_force) {
    lattice_t L;
    if (get_lattice(lattice, &L)) return ORACLE_BAD_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || (L.d == 2 && nz != 1)) return ORACLE_BAD_ARG;
    const int64_t n[3] = {nx, ny, nz};
    const int64_t N = nx * ny * nz;
    (void)force;
    for (int64_t node = 0; node < N; ++node) {
        if (wall && wall[node]) {
            lam_rho[node] = lam_rho_next[node];
            for (int i = 0; i < L.d; ++i) lam_u[i * N + node] = lam_u_next[i * N + node];
        } else {
            lam_rho[node] = 0.0;
            for (int i = 0; i < L.d; ++i) lam_u[i * N + node] = 0.0;
        }
    }
    for (int64_t node = 0; node < N; ++node) {
        if (wall && wall[node]) continue;
        const int64_t x[3] = {node % nx, (node / nx) % ny, node / (nx * ny)};
        /* forward recompute of this node's outputs */
        double rho_new = 0.0, mom[3] = {0.0, 0.0, 0.0};
        int64_t srcs[19];
        for (int a = 0; a < L.q; ++a) {
            int64_t y[3] = {0, 0, 0};
            for (int i = 0; i < 3; ++i) {
                y[i] = upstream(x[i], L.c[a][i], n[i], (periodic >> i) & 1u);
                if (y[i] < 0) return ORACLE_OUTSIDE;
            }
            srcs[a] = (y[2] * ny + y[1]) * nx + y[0];
            double ut[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < L.d; ++i) ut[i] = u[i * N + srcs[a]];
            const double f = feq(&L, a, rho[srcs[a]], ut);
            rho_new += f;
            for (int i = 0; i < L.d; ++i) mom[i] += (double)L.c[a][i] * f;
        }
        double lam_r = lam_rho_next[node];
        double lam_m[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < L.d; ++i) {
            const double lu = lam_u_next[i * N + node];
            lam_r -= lu * mom[i] / (rho_new * rho_new);
            lam_m[i] = lu / rho_new;
            if (grad_force) grad_force[i] += lu;
        }
        /* scatter back to the upstream sources */
        for (int a = 0; a < L.q; ++a) {
            const int64_t s = srcs[a];
            double ut[3] = {0.0, 0.0, 0.0}, cu = 0.0, uu = 0.0;
            for (int i = 0; i < L.d; ++i) {
                ut[i] = u[i * N + s];
                cu += (double)L.c[a][i] * ut[i];
                uu += ut[i] * ut[i];
            }
            double g = lam_r;
            for (int i = 0; i < L.d; ++i) g += (double)L.c[a][i] * lam_m[i];
            const double w = L.w[a];
            lam_rho[s] += g * w * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            for (int i = 0; i < L.d; ++i)
                lam_u[i * N + s] += g * w * rho[s] *
                                    (3.0 * L.c[a][i] + 9.0 * cu * L.c[a][i] - 3.0 * ut[i]);
        }
    }
    return ORACLE_OK;
}

/* Downstream coordinate x + c along one axis; -1 if it leaves a closed axis. */
static int64_t downstream(int64_t x, int c, int64_t n, int periodic) {
    int64_t y = x + c;
    if (y < 0 || y >= n) {
        if (!periodic) return -1;
        y = (y % n + n) % n;
    }
    return y;
}

/*
 * The same adjoint as oracle_adjoint_step, written as a gather so that the
 * node loops can run on several threads.  Pass 1 forms (lam_r, lam_m) of every
 * fluid node x exactly as oracle_adjoint_step does.  Pass 2 visits every source
 * node s and adds, for each direction a whose downstream node x = s + c_a is
 * fluid, the same term the scatter adds, in the scatter's order (ascending x,
 * then ascending a), starting from the same initial value.  Every lam value is
 * therefore the same sequence of operations on the same operands, and the
 * result is bitwise equal to oracle_adjoint_step's for any thread count.
 */
int oracle_adjoint_step_gather(int lattice, int64_t nx, int64_t ny, int64_t nz,
                               uint32_t periodic, const uint8_t *wall, const double *rho,
                               const double *u, const double *force,
                               const double *lam_rho_next, const double *lam_u_next,
                               double *lam_rho, double *lam_u, double *grad_force) {
    lattice_t L;
    if (get_lattice(lattice, &L)) return ORACLE_BAD_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || (L.d == 2 && nz != 1)) return ORACLE_BAD_ARG;
    const int64_t n[3] = {nx, ny, nz};
    const int64_t N = nx * ny * nz;
    (void)force;
    double *lr = (double *)malloc(sizeof(double) * (size_t)N);
    double *lm = (double *)malloc(sizeof(double) * (size_t)N * 3);
    if (!lr || !lm) { free(lr); free(lm); return ORACLE_NOMEM; }
    int outside = 0;
    /* pass 1: the adjoints of each fluid node's two outputs */
#pragma omp parallel for schedule(static)
    for (int64_t node = 0; node < N; ++node) {
        if (wall && wall[node]) continue;
        const int64_t x[3] = {node % nx, (node / nx) % ny, node / (nx * ny)};
        double rho_new = 0.0, mom[3] = {0.0, 0.0, 0.0};
        int bad = 0;
        for (int a = 0; a < L.q && !bad; ++a) {
            int64_t y[3] = {0, 0, 0};
            for (int i = 0; i < 3; ++i) {
                y[i] = upstream(x[i], L.c[a][i], n[i], (periodic >> i) & 1u);
                if (y[i] < 0) bad = 1;
            }
            if (bad) break;
            const int64_t src = (y[2] * ny + y[1]) * nx + y[0];
            double ut[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < L.d; ++i) ut[i] = u[i * N + src];
            const double f = feq(&L, a, rho[src], ut);
            rho_new += f;
            for (int i = 0; i < L.d; ++i) mom[i] += (double)L.c[a][i] * f;
        }
        if (bad) {
#pragma omp atomic write
            outside = 1;
            continue;
        }
        double lam_r = lam_rho_next[node];
        for (int i = 0; i < L.d; ++i) {
            const double lu = lam_u_next[i * N + node];
            lam_r -= lu * mom[i] / (rho_new * rho_new);
            lm[3 * node + i] = lu / rho_new;
        }
        lr[node] = lam_r;
    }
    if (outside) { free(lr); free(lm); return ORACLE_OUTSIDE; }
    /* d output / d force = identity on fluid nodes, summed in node order */
    if (grad_force)
        for (int64_t node = 0; node < N; ++node) {
            if (wall && wall[node]) continue;
            for (int i = 0; i < L.d; ++i) grad_force[i] += lam_u_next[i * N + node];
        }
    /* pass 2: every source gathers what the scatter would have sent it */
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        const int64_t y[3] = {s % nx, (s / nx) % ny, s / (nx * ny)};
        int64_t dst[19];
        int dir[19], k = 0;
        for (int a = 0; a < L.q; ++a) {
            int64_t x[3] = {0, 0, 0};
            int ok = 1;
            for (int i = 0; i < 3 && ok; ++i) {
                x[i] = downstream(y[i], L.c[a][i], n[i], (periodic >> i) & 1u);
                if (x[i] < 0) ok = 0;
            }
            if (!ok) continue;
            const int64_t xn = (x[2] * ny + x[1]) * nx + x[0];
            if (wall && wall[xn]) continue;
            /* insert (xn, a) keeping ascending (x, a) order */
            int j = k++;
            while (j > 0 && dst[j - 1] > xn) {
                dst[j] = dst[j - 1];
                dir[j] = dir[j - 1];
                --j;
            }
            dst[j] = xn;
            dir[j] = a;
        }
        double acc_r = (wall && wall[s]) ? lam_rho_next[s] : 0.0;
        double acc_u[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < L.d; ++i) acc_u[i] = (wall && wall[s]) ? lam_u_next[i * N + s] : 0.0;
        for (int t = 0; t < k; ++t) {
            const int a = dir[t];
            const int64_t xn = dst[t];
            double ut[3] = {0.0, 0.0, 0.0}, cu = 0.0, uu = 0.0;
            for (int i = 0; i < L.d; ++i) {
                ut[i] = u[i * N + s];
                cu += (double)L.c[a][i] * ut[i];
                uu += ut[i] * ut[i];
            }
            double g = lr[xn];
            for (int i = 0; i < L.d; ++i) g += (double)L.c[a][i] * lm[3 * xn + i];
            const double w = L.w[a];
            acc_r += g * w * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            for (int i = 0; i < L.d; ++i)
                acc_u[i] += g * w * rho[s] * (3.0 * L.c[a][i] + 9.0 * cu * L.c[a][i] - 3.0 * ut[i]);
        }
        lam_rho[s] = acc_r;
        for (int i = 0; i < L.d; ++i) lam_u[i * N + s] = acc_u[i];
    }
    free(lr);
    free(lm);
    return ORACLE_OK;
}

/*
 * The viscosity term of one reverse step.  Not in the paper: the chain rule of
 * the particle speed of Eq. (6).  nu enters a rollout only through
 * e = 6 nu / dx: initial and wall velocities are u / e in lattice units, the
 * force increment is g dx / e^2, the output velocity is e ut, and Eqs. (4)-(5)
 * themselves do not depend on e.  For one step from the state (rho, ut) this
 * returns sum over fluid nodes x of
 *     lam_rho_next(x) D_rho(x) + lam_u_next(x) . D_u(x),
 *     D_rho = -drho',  D_u = m'/rho' - (dm'/rho' - m' drho' / rho'^2) - force,
 * where rho', m' are the sums of Eqs. (4)-(5) and drho', dm' the same sums of
 * dF_a = d/d(eps) f_a^eq(rho, (1 + eps) ut) at eps = 0
 *      = w_a rho (3 c.ut + 9 (c.ut)^2 - 3 ut.ut).
 * Summed over the steps of a rollout with lam_next the adjoint of the state the
 * step produced, it gives e dL/de.  *status: ORACLE_OK or an error code.
 */
double oracle_nu_term(int lattice, int64_t nx, int64_t ny, int64_t nz, uint32_t periodic,
                      const uint8_t *wall, const double *rho, const double *u, const double *force,
                      const double *lam_rho_next, const double *lam_u_next, int *status) {
    lattice_t L;
    *status = ORACLE_OK;
    if (get_lattice(lattice, &L) || nx < 1 || ny < 1 || nz < 1 || (L.d == 2 && nz != 1)) {
        *status = ORACLE_BAD_ARG;
        return 0.0;
    }
    const int64_t n[3] = {nx, ny, nz};
    const int64_t N = nx * ny * nz;
    double total = 0.0;
    for (int64_t node = 0; node < N; ++node) {
        if (wall && wall[node]) continue;
        const int64_t x[3] = {node % nx, (node / nx) % ny, node / (nx * ny)};
        double r = 0.0, m[3] = {0.0, 0.0, 0.0}, dr = 0.0, dm[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < L.q; ++a) {
            int64_t y[3] = {0, 0, 0};
            for (int i = 0; i < 3; ++i) {
                y[i] = upstream(x[i], L.c[a][i], n[i], (periodic >> i) & 1u);
                if (y[i] < 0) { *status = ORACLE_OUTSIDE; return 0.0; }
            }
            const int64_t src = (y[2] * ny + y[1]) * nx + y[0];
            double ut[3] = {0.0, 0.0, 0.0}, cu = 0.0, uu = 0.0;
            for (int i = 0; i < L.d; ++i) {
                ut[i] = u[i * N + src];
                cu += (double)L.c[a][i] * ut[i];
                uu += ut[i] * ut[i];
            }
            const double f = feq(&L, a, rho[src], ut);
            const double df = L.w[a] * rho[src] * (3.0 * cu + 9.0 * cu * cu - 3.0 * uu);
            r += f;
            dr += df;
            for (int i = 0; i < L.d; ++i) {
                m[i] += (double)L.c[a][i] * f;
                dm[i] += (double)L.c[a][i] * df;
            }
        }
        double t = -lam_rho_next[node] * dr;
        for (int i = 0; i < L.d; ++i) {
            const double du = dm[i] / r - m[i] * dr / (r * r);
            const double Du = m[i] / r - du - (force ? force[i] : 0.0);
            t += lam_u_next[i * N + node] * Du;
        }
        total += t;
    }
    return total;
}
