/*
 * Plain FP64 CPU oracle of the two-phase weakly compressible SPH particle loop
 * (Wei et al., "Behavior of Oil under Breaking Waves by a Two-phase SPH
 * Model", Sec. II "Two-phase SPH model").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker for the CUDA
 * path: it is compiled and called by the test suite, by the smoke check and by
 * the benchmark's CPU-baseline leg, and by nothing else.  It shares no code,
 * header, table or helper with the CUDA library.  Every quantity is computed
 * in double precision, in the order the equations are written, with no
 * blocking, fusion or reordering.
 *
 * Notation follows the paper: rho density, P pressure, beta and gamma of the
 * equation of state, m particle mass, W the smoothing kernel, u velocity,
 * u_ij = u_i - u_j, r_ij = x_i - x_j, mu dynamic and nu kinematic viscosity,
 * alpha_s the interfacial tension coefficient, C the colour index,
 * sigma = rho/m the particle number density (called sigma_n here to keep it
 * apart from the tension coefficient), T the surface stress tensor.
 *
 * Readings where the paper is silent (each also stated where it is used):
 *   - W is the Wendland C2 kernel with support 2h.
 *   - j is a neighbour of i iff j != i and |r_ij|^2 < (2h)^2.
 *   - particle mass is a per-phase constant supplied by the caller.
 *   - dynamic boundary particles are phase 0 (water) everywhere.
 *   - the per-phase renormalisation (Eq. ct_dist_3) is a Jacobi update over
 *     same-phase neighbours including i itself, applied at stage 1 of every
 *     renorm_every-th step.  Dynamic boundary particles take it like water
 *     particles (renorm_walls = 1, the default): Sec. III gives them the
 *     fluid's equations of continuity and state, and Eq. ct_dist_3 belongs to
 *     the discretised continuity equation (Sec. II-B).  renorm_walls = 0 is a
 *     stabilisation of this library's long runs, not the paper's: boundary
 *     particles then keep the density continuity gives them while still
 *     entering the fluid's sums as water.  The colour gradient of the same
 *     stage uses the density that entered the stage (before
 *     renormalisation), everything after it uses the renormalised density.
 *   - T = 0 exactly when grad C = 0 (no threshold: |T| <= alpha_s |grad C|
 *     tends to zero with grad C).
 *   - time integration is the explicit midpoint predictor-corrector.
 *   - a periodic axis (the cross-tank boundary condition of the flume runs,
 *     Sec. "Laboratory experiment & numerical setup") is a box side of a
 *     whole number of cells; r_ij is taken as the minimum image along it and
 *     positions are wrapped into the box after every step.
 *   - the piston wavemaker (same section) is a set of boundary particles
 *     that move rigidly along one axis with a prescribed displacement X(t);
 *     the predictor puts them at X(t + dt/2) with velocity X'(t + dt/2) and
 *     the corrector at X(t + dt) with velocity X'(t + dt).  Like the other
 *     boundary particles their density integrates and their acceleration is
 *     not computed.
 *
 * Parity status: every function here is pinned by a CPU test (kernel
 * normalisation, partition of unity, EOS closed form, renormalisation
 * invariants, pairwise antisymmetry, brute-force neighbour sets, exact
 * kinematics, hydrostatic column, Laplace jump; periodic box against the
 * replicated box, translation invariance and the periodic lattice at rest;
 * the paper's wave-maker formula and exact piston kinematics).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t dim;          /* 2 or 3 */
    int32_t visc_form;    /* 0: dynamic form (Eq. visc_2), 1: kinematic form (Eq. visc_1) */
    int32_t renorm_every; /* Eq. ct_dist_3 at stage 1 of steps n % k == 0; 0 = never */
    int32_t periodic;     /* bit k set: axis k is periodic with period box_hi - box_lo */
    int32_t renorm_walls; /* 1: boundary particles are renormalised as water (Sec. II-B with
                             Sec. III); 0: they keep their continuity density */
    double h;             /* smoothing length */
    double c0;            /* reference speed of sound C_s0 */
    double gamma;         /* exponent of the equation of state */
    double delta;         /* regulariser of the viscous term, Eq. kvis */
    double alpha_s;       /* interfacial surface tension coefficient, Eq. csf */
    double cell_size;     /* edge of the cell grid used for the neighbour search */
    double g[3];          /* gravitational acceleration */
    double rho0[2];       /* reference density per phase (0 water, 1 oil) */
    double mu[2];         /* dynamic viscosity per phase */
    double mass[2];       /* particle mass per phase */
    double box_lo[3];
    double box_hi[3];
} or_params;

/* Prescribed piston motion along `axis`: for t <= t_end
 *   X(t) = sum_c amp_c (sin(omega_c t + phase_c) - sin(phase_c)),
 *   X'(t) = sum_c amp_c omega_c cos(omega_c t + phase_c);
 * after t_end the piston stays at X(t_end) with zero velocity.  The paper's
 * stroke x(t) = S/2 - S/2 cos(2 pi f t), 0 <= t <= 1/(2f), is one component
 * with amp = S/2, omega = 2 pi f, phase = -pi/2 and t_end = 1/(2f).        */
typedef struct {
    int32_t axis;
    int32_t ncomp;        /* 0..8; 0 = no motion */
    double t_end;
    double amp[8];
    double omega[8];
    double phase[8];
} or_piston;

double or_piston_disp(const or_piston *m, double t)
{
    double te = t < m->t_end ? t : m->t_end;
    double X = 0.0;
    for (int c = 0; c < m->ncomp; ++c) X += m->amp[c] * (sin(m->omega[c] * te + m->phase[c]) - sin(m->phase[c]));
    return X;
}

double or_piston_vel(const or_piston *m, double t)
{
    if (t > m->t_end) return 0.0;
    double U = 0.0;
    for (int c = 0; c < m->ncomp; ++c) U += m->amp[c] * m->omega[c] * cos(m->omega[c] * t + m->phase[c]);
    return U;
}

/* Period of axis k (0 when the axis is not periodic). */
static double period(const or_params *p, int k)
{
    return (p->periodic >> k) & 1 ? p->box_hi[k] - p->box_lo[k] : 0.0;
}

/* r_ij = x_i - x_j, minimum image along periodic axes; returns |r_ij|^2. */
static double pair_r(const or_params *p, const double *x, int64_t i, int64_t j, double *rij)
{
    double s = 0.0;
    for (int k = 0; k < p->dim; ++k) {
        double d = x[i * p->dim + k] - x[j * p->dim + k];
        double L = period(p, k);
        if (L > 0.0) d -= L * nearbyint(d / L);
        rij[k] = d;
        s += d * d;
    }
    return s;
}

/* Coordinate k of a position wrapped into [box_lo, box_hi) when axis k is
 * periodic; unchanged otherwise. */
static double wrapped(const or_params *p, int k, double v)
{
    double L = period(p, k);
    if (L > 0.0) v -= L * floor((v - p->box_lo[k]) / L);
    return v;
}

/* ------------------------------------------------------------------------ */
/* Smoothing kernel: Wendland C2, W(q) = alpha_d (1 - q/2)^4 (2q + 1), q=r/h */

static double wendland_alpha(int dim, double h)
{
    if (dim == 2) return 7.0 / (4.0 * M_PI * h * h);
    return 21.0 / (16.0 * M_PI * h * h * h);
}

double or_W(int dim, double h, double r)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return wendland_alpha(dim, h) * t * t * t * t * (2.0 * q + 1.0);
}

/* dW/dr = alpha_d * (-5 q / h) * (1 - q/2)^3 */
double or_dWdr(int dim, double h, double r)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return wendland_alpha(dim, h) * (-5.0 * q / h) * t * t * t;
}

/* grad_i W_ij = (dW/dr) r_ij / |r_ij|  (zero at r = 0) */
static void grad_W(int dim, double h, const double *rij, double r, double *out)
{
    for (int k = 0; k < 3; ++k) out[k] = 0.0;
    if (r <= 0.0) return;
    double f = or_dWdr(dim, h, r) / r;
    for (int k = 0; k < dim; ++k) out[k] = f * rij[k];
}

/* ------------------------------------------------------------------------ */
/* Equation of state, Eqs. state and beta: P = beta[(rho/rho0)^gamma - 1],
 * beta = rho0 C_s0^2 / gamma.                                               */

double or_eos(const or_params *p, int phase, double rho)
{
    double rho0 = p->rho0[phase];
    double beta = rho0 * p->c0 * p->c0 / p->gamma;
    return beta * (pow(rho / rho0, p->gamma) - 1.0);
}

/* Inverse of the equation of state: the density at which P = pressure. */
double or_eos_inverse(const or_params *p, int phase, double pressure)
{
    double rho0 = p->rho0[phase];
    double beta = rho0 * p->c0 * p->c0 / p->gamma;
    return rho0 * pow(1.0 + pressure / beta, 1.0 / p->gamma);
}

/* ------------------------------------------------------------------------ */
/* Cell grid used by the neighbour search.  A cell is the integer part of
 * (x - box_lo) / cell_size on each axis (x wrapped into the box along a
 * periodic axis); the grid has floor((box_hi - box_lo) / cell_size) + 1
 * cells per axis, or (box_hi - box_lo) / cell_size rounded along a periodic
 * axis, and the linear id is ix + nx * (iy + ny * iz).                      */

void or_grid_dims(const or_params *p, int32_t *dims)
{
    for (int k = 0; k < 3; ++k) dims[k] = 1;
    for (int k = 0; k < p->dim; ++k) {
        double m = (p->box_hi[k] - p->box_lo[k]) / p->cell_size;
        dims[k] = period(p, k) > 0.0 ? (int32_t)nearbyint(m) : (int32_t)floor(m) + 1;
    }
}

/* Returns the number of particles outside the box (their id is -1). */
int64_t or_cell_ids(const or_params *p, int64_t n, const double *x, int32_t *cell)
{
    int32_t dims[3];
    or_grid_dims(p, dims);
    int64_t outside = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t c[3] = {0, 0, 0};
        int ok = 1;
        for (int k = 0; k < p->dim; ++k) {
            double s = floor((wrapped(p, k, x[i * p->dim + k]) - p->box_lo[k]) / p->cell_size);
            if (period(p, k) > 0.0 && s >= (double)dims[k]) s = dims[k] - 1;  /* rounding at box_hi */
            if (!(s >= 0.0 && s < (double)dims[k])) ok = 0;
            else c[k] = (int32_t)s;
        }
        if (!ok) { cell[i] = -1; ++outside; continue; }
        cell[i] = c[0] + dims[0] * (c[1] + dims[1] * c[2]);
    }
    return outside;
}

/* Permutation that orders particles by (cell id, particle index): perm[k]
 * is the index of the k-th particle in that order.                         */
static const int32_t *g_sort_cell;
static int cmp_cell_then_index(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    if (g_sort_cell[i] != g_sort_cell[j]) return g_sort_cell[i] < g_sort_cell[j] ? -1 : 1;
    return (i > j) - (i < j);
}

void or_sort_perm(int64_t n, const int32_t *cell, int64_t *perm)
{
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    g_sort_cell = cell;
    qsort(perm, (size_t)n, sizeof(int64_t), cmp_cell_then_index);
    g_sort_cell = NULL;
}

/* ------------------------------------------------------------------------ */
/* Neighbour sets.  j is a neighbour of i iff j != i and |x_i - x_j|^2 < (2h)^2.
 * Results are in CSR form: start[i] .. start[i+1] index list[], each row in
 * ascending j.  Both functions return the number of entries, or -1 when the
 * caller's list capacity is too small (start[] is then still filled).      */

static double dist2(const or_params *p, const double *x, int64_t i, int64_t j)
{
    double rij[3];
    return pair_r(p, x, i, j, rij);
}

int64_t or_neighbours_brute(const or_params *p, int64_t n, const double *x,
                            int64_t *start, int32_t *list, int64_t cap)
{
    double R2 = 4.0 * p->h * p->h;
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        start[i] = total;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i || dist2(p, x, i, j) >= R2) continue;
            if (total < cap) list[total] = (int32_t)j;
            ++total;
        }
    }
    start[n] = total;
    return total <= cap ? total : -1;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Same sets through a cell list: particles sorted by cell, every i scans the
 * cells within w = ceil(2h / cell_size) of its own on each axis (wrapping
 * around a periodic axis).  Returns -3 when a periodic axis has fewer than
 * 2w + 1 cells.                                                             */
int64_t or_neighbours_cells(const or_params *p, int64_t n, const double *x,
                            int64_t *start, int32_t *list, int64_t cap)
{
    int32_t dims[3];
    or_grid_dims(p, dims);
    int64_t ncell = (int64_t)dims[0] * dims[1] * dims[2];
    int32_t *cell = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int64_t *perm = malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    int64_t *cstart = calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *count = malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    if (or_cell_ids(p, n, x, cell) != 0) {
        free(cell); free(perm); free(cstart); free(count);
        return -2;
    }
    or_sort_perm(n, cell, perm);
    for (int64_t i = 0; i < n; ++i) cstart[cell[i] + 1]++;
    for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    double R2 = 4.0 * p->h * p->h;
    int dim = p->dim;
    const int w = (int)ceil(2.0 * p->h / p->cell_size);
    const int wz = dim == 3 ? w : 0;
    /* a periodic axis needs 2w + 1 distinct cells, else a cell would be
     * scanned twice */
    int per[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
        per[k] = period(p, k) > 0.0;
        if (per[k] && dims[k] < 2 * w + 1) {
            free(cell); free(perm); free(cstart); free(count);
            return -3;
        }
    }

    /* pass 1: counts */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int32_t ci = cell[i];
        int32_t cx = ci % dims[0], cy = (ci / dims[0]) % dims[1], cz = ci / (dims[0] * dims[1]);
        int64_t cnt = 0;
        for (int dz = -wz; dz <= wz; ++dz)
            for (int dy = -w; dy <= w; ++dy)
                for (int dx = -w; dx <= w; ++dx) {
                    int32_t X = cx + dx, Y = cy + dy, Z = cz + dz;
                    if (per[0]) X = (X + dims[0]) % dims[0];
                    if (per[1]) Y = (Y + dims[1]) % dims[1];
                    if (per[2]) Z = (Z + dims[2]) % dims[2];
                    if (X < 0 || Y < 0 || Z < 0 || X >= dims[0] || Y >= dims[1] || Z >= dims[2]) continue;
                    int64_t c = X + (int64_t)dims[0] * (Y + (int64_t)dims[1] * Z);
                    for (int64_t k = cstart[c]; k < cstart[c + 1]; ++k) {
                        int64_t j = perm[k];
                        if (j != i && dist2(p, x, i, j) < R2) ++cnt;
                    }
                }
        count[i] = cnt;
    }
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) { start[i] = total; total += count[i]; }
    start[n] = total;
    if (total > cap) {
        free(cell); free(perm); free(cstart); free(count);
        return -1;
    }
    /* pass 2: fill and order each row by j */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int32_t ci = cell[i];
        int32_t cx = ci % dims[0], cy = (ci / dims[0]) % dims[1], cz = ci / (dims[0] * dims[1]);
        int64_t wr = start[i];
        for (int dz = -wz; dz <= wz; ++dz)
            for (int dy = -w; dy <= w; ++dy)
                for (int dx = -w; dx <= w; ++dx) {
                    int32_t X = cx + dx, Y = cy + dy, Z = cz + dz;
                    if (per[0]) X = (X + dims[0]) % dims[0];
                    if (per[1]) Y = (Y + dims[1]) % dims[1];
                    if (per[2]) Z = (Z + dims[2]) % dims[2];
                    if (X < 0 || Y < 0 || Z < 0 || X >= dims[0] || Y >= dims[1] || Z >= dims[2]) continue;
                    int64_t c = X + (int64_t)dims[0] * (Y + (int64_t)dims[1] * Z);
                    for (int64_t k = cstart[c]; k < cstart[c + 1]; ++k) {
                        int64_t j = perm[k];
                        if (j != i && dist2(p, x, i, j) < R2) list[wr++] = (int32_t)j;
                    }
                }
        qsort(list + start[i], (size_t)(start[i + 1] - start[i]), sizeof(int32_t), cmp_i32);
    }
    free(cell); free(perm); free(cstart); free(count);
    return total;
}

/* Builds the neighbour CSR into freshly allocated arrays (caller frees). */
static int build_neighbours(const or_params *p, int64_t n, const double *x,
                            int64_t **start_out, int32_t **list_out)
{
    int64_t *start = malloc(sizeof(int64_t) * (size_t)(n + 1));
    /* first call with zero capacity only sizes the lists */
    int64_t cap = 0;
    int64_t r = or_neighbours_cells(p, n, x, start, NULL, 0);
    if (r == -2 || r == -3) { free(start); return (int)r; }
    cap = start[n];
    int32_t *list = malloc(sizeof(int32_t) * (size_t)(cap ? cap : 1));
    r = or_neighbours_cells(p, n, x, start, list, cap);
    if (r < 0) { free(start); free(list); return (int)r; }
    *start_out = start;
    *list_out = list;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Harmonic-mean viscosities (Sec. II-C): mu_ij = 2 mu_i mu_j / (mu_i + mu_j),
 * nu_ij likewise with nu = mu / rho0 per phase.                            */

static double harmonic(double a, double b)
{
    return 2.0 * a * b / (a + b);
}

/* ------------------------------------------------------------------------ */
/* One evaluation of the rates at state (x, u, rho_in).
 *
 * Outputs (all length n, vectors n*dim, tensors n*dim*dim row-major):
 *   rho    density after the optional per-phase renormalisation (Eq. ct_dist_3)
 *   P      pressure, Eq. state
 *   gradC  colour-index gradient, Eq. cd
 *   T      surface stress tensor, Eq. csf
 *   a      acceleration Du/Dt: pressure (Eq. dist_p_1) + viscosity
 *          (Eq. visc_2 or visc_1) + surface tension (F_s/rho) + g; zero for
 *          dynamic boundary particles, whose motion is prescribed
 *   drho   density rate, Eq. ct_dist_2, for every particle
 * Returns 0, or -2 when a particle is outside the box.                     */
int or_eval(const or_params *p, int64_t n, const double *x, const double *u,
            const double *rho_in, const uint8_t *phase, const uint8_t *wall,
            int renorm, double *rho, double *P, double *gradC, double *T,
            double *a, double *drho)
{
    const int d = p->dim;
    int64_t *start = NULL;
    int32_t *list = NULL;
    int rc = build_neighbours(p, n, x, &start, &list);
    if (rc != 0) return rc;

    /* Eq. ct_dist_3: rho_i = sum_{same phase} m_j W_ij / sum_{same phase} (m_j/rho_j) W_ij,
     * the sums running over i itself and its same-phase neighbours.  Boundary
     * particles (wall != 0, water) are renormalised like water particles when
     * renorm_walls is set: they share the fluid's continuity equation
     * (Sec. III), of whose discretisation Eq. ct_dist_3 is part (Sec. II-B);
     * otherwise they keep the density continuity gives them. */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (!renorm || (wall[i] && !p->renorm_walls)) { rho[i] = rho_in[i]; continue; }
        int ph = phase[i];
        double num = p->mass[ph] * or_W(d, p->h, 0.0);
        double den = p->mass[ph] / rho_in[i] * or_W(d, p->h, 0.0);
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            int64_t j = list[k];
            if (phase[j] != ph) continue;
            double r = sqrt(dist2(p, x, i, j));
            double Wij = or_W(d, p->h, r);
            num += p->mass[phase[j]] * Wij;
            den += p->mass[phase[j]] / rho_in[j] * Wij;
        }
        rho[i] = num / den;
    }

    /* Eq. cd with C_i^y = 0 and C_j^y = 1 for j of the other phase:
     * grad C_i = sigma_i sum_{j other phase} (1/sigma_j^2) grad_i W_ij,
     * sigma = rho/m with the density that entered this stage.
     * Then Eq. csf: T = alpha_s / |grad C| (|grad C|^2 / d I - grad C (x) grad C). */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double gc[3] = {0.0, 0.0, 0.0};
        double sigma_i = rho_in[i] / p->mass[phase[i]];
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            int64_t j = list[k];
            if (phase[j] == phase[i]) continue;
            double rij[3], gw[3];
            double r = sqrt(pair_r(p, x, i, j, rij));
            grad_W(d, p->h, rij, r, gw);
            double sigma_j = rho_in[j] / p->mass[phase[j]];
            for (int c = 0; c < d; ++c) gc[c] += sigma_i * (1.0 / (sigma_j * sigma_j)) * gw[c];
        }
        double norm2 = 0.0;
        for (int c = 0; c < d; ++c) {
            gradC[i * d + c] = gc[c];
            norm2 += gc[c] * gc[c];
        }
        double norm = sqrt(norm2);
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) {
                double v = 0.0;
                if (norm > 0.0)
                    v = p->alpha_s / norm * ((r == c ? norm2 / d : 0.0) - gc[r] * gc[c]);
                T[(i * d + r) * d + c] = v;
            }
    }

    /* Eq. state on the (renormalised) density. */
    for (int64_t i = 0; i < n; ++i) P[i] = or_eos(p, phase[i], rho[i]);

#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int pi = phase[i];
        double m_i = p->mass[pi];
        double sigma_i = rho[i] / m_i;
        double acc[3] = {0.0, 0.0, 0.0};
        double visc[3] = {0.0, 0.0, 0.0};
        double st[3] = {0.0, 0.0, 0.0};
        double div = 0.0;
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            int64_t j = list[k];
            int pj = phase[j];
            double m_j = p->mass[pj];
            double rij[3] = {0, 0, 0}, uij[3] = {0, 0, 0}, gw[3];
            for (int c = 0; c < d; ++c) uij[c] = u[i * d + c] - u[j * d + c];
            double r2 = pair_r(p, x, i, j, rij);
            double r = sqrt(r2);
            grad_W(d, p->h, rij, r, gw);
            double rdotgw = 0.0, udotgw = 0.0;
            for (int c = 0; c < d; ++c) {
                rdotgw += rij[c] * gw[c];
                udotgw += uij[c] * gw[c];
            }

            /* Eq. dist_p_1: -sum m_j (P_i/rho_i^2 + P_j/rho_j^2) grad_i W_ij */
            double pterm = m_j * (P[i] / (rho[i] * rho[i]) + P[j] / (rho[j] * rho[j]));
            for (int c = 0; c < d; ++c) acc[c] -= pterm * gw[c];

            /* Eq. visc_2 (dynamic): (1/rho_i) sum 2 mu_ij (m_j/rho_j) (r.gradW)/(r^2+delta^2) u_ij
             * Eq. visc_1 (kinematic): sum 2 nu_ij (m_j/rho_j) (r.gradW)/(r^2+delta^2) u_ij */
            double coef;
            if (p->visc_form == 0) {
                double mu_ij = harmonic(p->mu[pi], p->mu[pj]);
                coef = (1.0 / rho[i]) * 2.0 * mu_ij * (m_j / rho[j]) * rdotgw / (r2 + p->delta * p->delta);
            } else {
                double nu_ij = harmonic(p->mu[pi] / p->rho0[pi], p->mu[pj] / p->rho0[pj]);
                coef = 2.0 * nu_ij * (m_j / rho[j]) * rdotgw / (r2 + p->delta * p->delta);
            }
            for (int c = 0; c < d; ++c) visc[c] += coef * uij[c];

            /* (F_s/rho)_i = (1/m_i) sum (T_i/sigma_i^2 + T_j/sigma_j^2) . grad_i W_ij */
            double sigma_j = rho[j] / m_j;
            for (int r_ = 0; r_ < d; ++r_) {
                double s = 0.0;
                for (int c = 0; c < d; ++c)
                    s += (T[(i * d + r_) * d + c] / (sigma_i * sigma_i) +
                          T[(j * d + r_) * d + c] / (sigma_j * sigma_j)) * gw[c];
                st[r_] += s / m_i;
            }

            /* Eq. ct_dist_2: rho_i sum (m_j/rho_j) u_ij . grad_i W_ij */
            div += (m_j / rho[j]) * udotgw;
        }
        drho[i] = rho[i] * div;
        for (int c = 0; c < d; ++c)
            a[i * d + c] = wall[i] ? 0.0 : acc[c] + visc[c] + st[c] + p->g[c];
    }
    free(start);
    free(list);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One predictor-corrector (explicit midpoint) step of size dt from time t,
 * in place.
 *   stage 1 at (x^n, u^n, rho^n), with the renormalisation when
 *     renorm_every > 0 and step_index % renorm_every == 0 (the renormalised
 *     density replaces rho^n);
 *   x* = x^n + dt/2 u^n, u* = u^n + dt/2 a^n, rho* = rho^n + dt/2 Drho^n;
 *   stage 2 at (x*, u*, rho*);
 *   x^{n+1} = x^n + dt u*, u^{n+1} = u^n + dt a*, rho^{n+1} = rho^n + dt Drho*.
 * Boundary particles (wall 1) keep x and u; piston particles (wall 2) move
 * with the prescribed motion m (NULL: at rest, like wall 1); the density of
 * both integrates.  Positions are then wrapped along periodic axes.
 * Returns 0, or -2 when a particle left the box.                           */
int or_step(const or_params *p, int64_t n, double *x, double *u, double *rho,
            const uint8_t *phase, const uint8_t *wall, double dt, int64_t step_index,
            const or_piston *m, double t)
{
    const int d = p->dim;
    size_t nv = (size_t)n * d, nt = (size_t)n * d * d;
    double *rho_s = malloc(sizeof(double) * n), *P = malloc(sizeof(double) * n);
    double *gc = malloc(sizeof(double) * nv), *T = malloc(sizeof(double) * nt);
    double *a = malloc(sizeof(double) * nv), *dr = malloc(sizeof(double) * n);
    double *xs = malloc(sizeof(double) * nv), *us = malloc(sizeof(double) * nv);
    double *rs = malloc(sizeof(double) * n);
    int renorm = p->renorm_every > 0 && step_index % p->renorm_every == 0;
    int moving = m != NULL && m->ncomp > 0;
    /* piston displacement over each stage and its velocity at the stage end */
    double X0 = moving ? or_piston_disp(m, t) : 0.0;
    double dX_half = moving ? or_piston_disp(m, t + 0.5 * dt) - X0 : 0.0;
    double dX_full = moving ? or_piston_disp(m, t + dt) - X0 : 0.0;
    double U_half = moving ? or_piston_vel(m, t + 0.5 * dt) : 0.0;
    double U_full = moving ? or_piston_vel(m, t + dt) : 0.0;

    int rc = or_eval(p, n, x, u, rho, phase, wall, renorm, rho_s, P, gc, T, a, dr);
    if (rc == 0) {
        for (int64_t i = 0; i < n; ++i) {
            rho[i] = rho_s[i];
            rs[i] = rho[i] + 0.5 * dt * dr[i];
            for (int c = 0; c < d; ++c) {
                size_t k = (size_t)i * d + c;
                if (wall[i] == 2 && moving) {
                    xs[k] = c == m->axis ? x[k] + dX_half : x[k];
                    us[k] = c == m->axis ? U_half : 0.0;
                } else {
                    xs[k] = wall[i] ? x[k] : x[k] + 0.5 * dt * u[k];
                    us[k] = wall[i] ? u[k] : u[k] + 0.5 * dt * a[k];
                }
            }
        }
        rc = or_eval(p, n, xs, us, rs, phase, wall, 0, rho_s, P, gc, T, a, dr);
    }
    if (rc == 0) {
        for (int64_t i = 0; i < n; ++i) {
            rho[i] = rho[i] + dt * dr[i];
            for (int c = 0; c < d; ++c) {
                size_t k = (size_t)i * d + c;
                if (wall[i] == 2 && moving) {
                    if (c == m->axis) x[k] = x[k] + dX_full;
                    u[k] = c == m->axis ? U_full : 0.0;
                } else if (!wall[i]) {
                    x[k] = x[k] + dt * us[k];
                    u[k] = u[k] + dt * a[k];
                }
                x[k] = wrapped(p, c, x[k]);
            }
        }
    }
    free(rho_s); free(P); free(gc); free(T); free(a); free(dr);
    free(xs); free(us); free(rs);
    return rc;
}

/* nsteps steps from time t0; the time advances by repeated addition of dt. */
int or_run(const or_params *p, int64_t n, double *x, double *u, double *rho,
           const uint8_t *phase, const uint8_t *wall, double dt,
           int64_t first_step, int64_t nsteps, const or_piston *m, double t0)
{
    double t = t0;
    for (int64_t s = 0; s < nsteps; ++s) {
        int rc = or_step(p, n, x, u, rho, phase, wall, dt, first_step + s, m, t);
        if (rc != 0) return rc;
        t += dt;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics over the fluid particles (dynamic boundary particles excluded):
 * out[0]      total mass
 * out[1..3]   linear momentum sum m u
 * out[4]      kinetic energy sum m |u|^2 / 2
 * out[5]      potential energy -sum m g.x
 * out[6..8]   centroid of the oil particles
 * out[9]      sphericity of the oil particles: sqrt(lambda_min / lambda_max)
 *             of the covariance of their positions (1 for a circle/sphere)
 * out[10]     max |u| over fluid particles
 * out[11]     number of oil particles                                      */

static void sym_eigen_minmax(int d, const double *A, double *lmin, double *lmax)
{
    if (d == 2) {
        double tr = A[0] + A[3], det = A[0] * A[3] - A[1] * A[2];
        double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));
        *lmin = 0.5 * tr - disc;
        *lmax = 0.5 * tr + disc;
        return;
    }
    /* cyclic Jacobi rotations on a 3x3 symmetric matrix */
    double M[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[r][c] = A[r * 3 + c];
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = M[0][1] * M[0][1] + M[0][2] * M[0][2] + M[1][2] * M[1][2];
        if (off < 1e-30 * (M[0][0] * M[0][0] + M[1][1] * M[1][1] + M[2][2] * M[2][2] + 1e-300)) break;
        for (int pq = 0; pq < 3; ++pq) {
            int P_ = pq == 2 ? 1 : 0, Q = pq == 0 ? 1 : 2;
            if (M[P_][Q] == 0.0) continue;
            double theta = 0.5 * atan2(2.0 * M[P_][Q], M[Q][Q] - M[P_][P_]);
            double c = cos(theta), s = sin(theta);
            for (int k = 0; k < 3; ++k) {
                double mkp = M[k][P_], mkq = M[k][Q];
                M[k][P_] = c * mkp - s * mkq;
                M[k][Q] = s * mkp + c * mkq;
            }
            for (int k = 0; k < 3; ++k) {
                double mpk = M[P_][k], mqk = M[Q][k];
                M[P_][k] = c * mpk - s * mqk;
                M[Q][k] = s * mpk + c * mqk;
            }
        }
    }
    double e0 = M[0][0], e1 = M[1][1], e2 = M[2][2];
    *lmin = fmin(e0, fmin(e1, e2));
    *lmax = fmax(e0, fmax(e1, e2));
}

void or_diag(const or_params *p, int64_t n, const double *x, const double *u,
             const uint8_t *phase, const uint8_t *wall, double *out)
{
    const int d = p->dim;
    for (int k = 0; k < 12; ++k) out[k] = 0.0;
    double cen[3] = {0, 0, 0};
    int64_t noil = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (wall[i]) continue;
        double m = p->mass[phase[i]];
        double u2 = 0.0;
        out[0] += m;
        for (int c = 0; c < d; ++c) {
            out[1 + c] += m * u[i * d + c];
            u2 += u[i * d + c] * u[i * d + c];
            out[5] -= m * p->g[c] * x[i * d + c];
        }
        out[4] += 0.5 * m * u2;
        if (sqrt(u2) > out[10]) out[10] = sqrt(u2);
        if (phase[i] == 1) {
            ++noil;
            for (int c = 0; c < d; ++c) cen[c] += x[i * d + c];
        }
    }
    out[11] = (double)noil;
    if (noil == 0) return;
    for (int c = 0; c < d; ++c) {
        cen[c] /= (double)noil;
        out[6 + c] = cen[c];
    }
    double cov[9] = {0};
    for (int64_t i = 0; i < n; ++i) {
        if (wall[i] || phase[i] != 1) continue;
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c)
                cov[r * d + c] += (x[i * d + r] - cen[r]) * (x[i * d + c] - cen[c]);
    }
    for (int k = 0; k < d * d; ++k) cov[k] /= (double)noil;
    double lmin, lmax;
    sym_eigen_minmax(d, cov, &lmin, &lmax);
    out[9] = lmax > 0.0 ? sqrt(fmax(lmin, 0.0) / lmax) : 0.0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
