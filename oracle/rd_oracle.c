/*
 * rd_oracle.c -- plain FP64, single-threaded CPU reference stepper.
 *
 * TEST INFRASTRUCTURE ONLY (see rd_oracle.h).  Written for readability, not
 * speed: one naive loop nest per pass, every neighbour fetched through a
 * boundary-aware accessor.
 */
#include "rd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int64_t lin(const orc_problem* p, int x, int y, int z)
{
    return ((int64_t)z * p->ny + y) * p->nx + x;
}

/* Index along one axis of extent n after applying the boundary rule of the
 * face that was crossed.  Only distance-1 ghosts are ever requested. */
static int ghost_index(int i, int n, int kind_lo, int kind_hi)
{
    if (i < 0) {
        if (kind_lo == ORC_PERIODIC) return i + n;
        return 0;                    /* zero flux (and held layers): c(-1) = c(0) */
    }
    if (i >= n) {
        if (kind_hi == ORC_PERIODIC) return i - n;
        return n - 1;
    }
    return i;
}

/* Value of field f (one species plane-stack) at (x,y,z) shifted by one cell
 * along ``axis`` in direction ``dir`` (-1/+1), honouring the boundary kinds
 * of species s. */
static double nb(const orc_problem* p, const double* f, int s,
                 int x, int y, int z, int axis, int dir)
{
    int X = x, Y = y, Z = z;
    if (axis == 0) X = ghost_index(x + dir, p->nx, p->bc[s][0], p->bc[s][1]);
    if (axis == 1) Y = ghost_index(y + dir, p->ny, p->bc[s][2], p->bc[s][3]);
    if (axis == 2) Z = ghost_index(z + dir, p->nz, p->bc[s][4], p->bc[s][5]);
    return f[lin(p, X, Y, Z)];
}

/* Second difference along one axis, divided by h^2. */
static double second_diff(const orc_problem* p, const double* f, int s,
                          int x, int y, int z, int axis)
{
    double c = f[lin(p, x, y, z)];
    double m = nb(p, f, s, x, y, z, axis, -1);
    double q = nb(p, f, s, x, y, z, axis, +1);
    return (m + q - 2.0 * c) / (p->h * p->h);
}

/* Weights T_pqr of eq. (4), indexed [r+1][q+1][p+1]: the planes r = -1 and
 * r = +1 hold the "plus" matrix, the plane r = 0 the matrix with -24 in its
 * centre. */
static const double T19[3][3][3] = {
    /* r = -1 */ {{0, 1, 0}, {1, 2, 1}, {0, 1, 0}},
    /* r =  0 */ {{1, 2, 1}, {2, -24, 2}, {1, 2, 1}},
    /* r = +1 */ {{0, 1, 0}, {1, 2, 1}, {0, 1, 0}},
};

/* Value at (x+dx, y+dy, z+dz), each shifted axis mapped through its own
 * boundary rule in turn (edge ghosts are composed from the face rules). */
static double nb3(const orc_problem* p, const double* f, int s,
                  int x, int y, int z, int dx, int dy, int dz)
{
    int X = ghost_index(x + dx, p->nx, p->bc[s][0], p->bc[s][1]);
    int Y = ghost_index(y + dy, p->ny, p->bc[s][2], p->bc[s][3]);
    int Z = ghost_index(z + dz, p->nz, p->bc[s][4], p->bc[s][5]);
    return f[lin(p, X, Y, Z)];
}

/* Eq. (3): the 19-point Laplacian, (1 / 6h^2) sum_pqr T_pqr c_{i+p,j+q,k+r}. */
static double laplacian19(const orc_problem* p, const double* f, int s,
                          int x, int y, int z)
{
    double acc = 0.0;
    for (int r = -1; r <= 1; ++r)
        for (int q = -1; q <= 1; ++q)
            for (int pp = -1; pp <= 1; ++pp) {
                double w = T19[r + 1][q + 1][pp + 1];
                if (w != 0.0) acc += w * nb3(p, f, s, x, y, z, pp, q, r);
            }
    return acc / (6.0 * p->h * p->h);
}

static double laplacian(const orc_problem* p, const double* f, int s,
                        int x, int y, int z)
{
    if (p->stencil == 19) return laplacian19(p, f, s, x, y, z);
    return second_diff(p, f, s, x, y, z, 0) + second_diff(p, f, s, x, y, z, 1)
         + second_diff(p, f, s, x, y, z, 2);
}

/* Velocity (u_x, u_y, u_z) of ORC_WIND_3D at time t. */
static void wind3(const orc_problem* p, double t, double u[3])
{
    u[0] = p->w3[0];
    u[1] = p->w3[1];
    u[2] = p->w3[2] * sin(t / p->w3[3]);
}

/* First-order upwind term -u d c / d(axis) at one cell: the backward
 * difference for u > 0, the forward one for u < 0 (Section 4.1). */
static double upwind(const orc_problem* p, const double* f, int s, int x, int y, int z,
                     int axis, double u)
{
    const double c = f[lin(p, x, y, z)];
    if (u > 0.0) return -u * (c - nb(p, f, s, x, y, z, axis, -1)) / p->h;
    if (u < 0.0) return -u * (nb(p, f, s, x, y, z, axis, +1) - c) / p->h;
    return 0.0;
}

double orc_wind(const orc_problem* p, int z)
{
    if (p->wind_kind == ORC_WIND_3D) return p->w3[0];
    if (p->wind_kind == ORC_WIND_LOG)
        return p->wind_u0 * log(1.0 + (double)z) / log(1.0 + (double)p->nz);
    if (p->wind_kind == ORC_WIND_CONST) return p->wind_u0;
    return 0.0;
}

/* Is (x,y,z) in a held (Dirichlet) boundary layer of species s?  Returns the
 * face index (0..5) or -1.  Faces are checked in the order -x,+x,-y,+y,-z,+z. */
static int held_face(const orc_problem* p, int s, int x, int y, int z)
{
    const int coord[3] = {x, y, z};
    const int ext[3] = {p->nx, p->ny, p->nz};
    for (int f = 0; f < 6; ++f) {
        if (p->bc[s][f] != ORC_DIRICHLET) continue;
        int axis = f / 2;
        int at = (f % 2 == 0) ? 0 : ext[axis] - 1;
        if (coord[axis] == at) return f;
    }
    return -1;
}

static int check(const orc_problem* p)
{
    if (!p) return -1;
    if (p->nx < 2 || p->ny < 2 || p->nz < 2) return -1;
    if (p->ns < 1 || p->ns > ORC_MAXS) return -1;
    if (!(p->h > 0.0) || !(p->dt > 0.0)) return -1;
    if (p->wind_kind == ORC_WIND_3D && !(p->w3[3] != 0.0)) return -1;
    for (int s = 0; s < p->ns; ++s)
        for (int a = 0; a < 3; ++a)
            if ((p->bc[s][2 * a] == ORC_PERIODIC) != (p->bc[s][2 * a + 1] == ORC_PERIODIC))
                return -1;
    if (p->stencil != 0 && p->stencil != 7 && p->stencil != 19) return -1;
    if (p->stencil == 19)   /* eq. (3) has one diffusivity per species */
        for (int s = 0; s < p->ns; ++s)
            if (p->D[s][1] != p->D[s][0] || p->D[s][2] != p->D[s][0]) return -1;
    switch (p->model) {
    case ORC_DIFFUSION: break;
    case ORC_BRUSSELATOR: if (p->ns != 2) return -1; break;
    case ORC_CH_FRONT: if (p->ns != 3) return -1; break;
    case ORC_AIR: if (p->ns != 3) return -1; break;
    case ORC_TURING: if (p->ns != 2) return -1; break;
    case ORC_CH_TABLE1: if (p->ns != 3) return -1; break;
    default: return -1;
    }
    return 0;
}

/* Reaction rates R(c) of eq. (1) for one cell, species values v[0..ns-1]. */
static void reaction(const orc_problem* p, const double* v, double* r)
{
    for (int s = 0; s < p->ns; ++s) r[s] = 0.0;
    switch (p->model) {
    case ORC_BRUSSELATOR: {
        /* du/dt = a - (b+1) u + u^2 v ;  dv/dt = b u - u^2 v */
        double a = p->p[0], b = p->p[1], u = v[0], w = v[1];
        r[0] = a - (b + 1.0) * u + u * u * w;
        r[1] = b * u - u * u * w;
        break;
    }
    case ORC_CH_FRONT: {
        /* a + b -> c at rate k a b (mass action) */
        double k = p->p[0];
        double q = k * v[0] * v[1];
        r[0] = -q;
        r[1] = -q;
        r[2] = q;
        break;
    }
    case ORC_AIR: {
        /* NO2 -> NO + O3 (rate j NO2);  NO + O3 -> NO2 (rate k NO O3);
         * species order NO, NO2, O3 */
        double j = p->p[0], k = p->p[1];
        double ph = j * v[1];
        double ti = k * v[0] * v[2];
        r[0] = ph - ti;
        r[1] = -ph + ti;
        r[2] = ph - ti;
        break;
    }
    case ORC_CH_TABLE1: {
        /* Table 1, row 3: c1 + c2 -> c3 at rate k1 c1 c2, and the sink
         * k2 c1 c3 of c1 and c3 (redissolution by the excess of c1) */
        double k1 = p->p[0], k2 = p->p[1];
        double c1 = v[0], c2 = v[1], c3 = v[2];
        r[0] = -k1 * c1 * c2 - k2 * c1 * c3;
        r[1] = -k1 * c1 * c2;
        r[2] = k1 * c1 * c2 - k2 * c1 * c3;
        break;
    }
    case ORC_TURING: {
        /* activator-inhibitor pair of Table 1, row 2:
         * dc1/dt = c1 - c1^3 - c2 ;  dc2/dt = gamma (c1 - alpha c2 - beta) */
        double alpha = p->p[0], beta = p->p[1], gamma = p->p[2];
        double c1 = v[0], c2 = v[1];
        r[0] = c1 - c1 * c1 * c1 - c2;
        r[1] = gamma * (c1 - alpha * c2 - beta);
        break;
    }
    default: break;
    }
}

/* One forward-Euler step from cur to nxt (Table 3), step index n. */
static void step(const orc_problem* p, double* cur, double* nxt, double* mu, int64_t n)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz, ns = p->ns;
    const int64_t nc = (int64_t)nx * ny * nz;

    /* boundary points: held layers take their value before the step */
    for (int s = 0; s < ns; ++s)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int f = held_face(p, s, x, y, z);
                    if (f >= 0) cur[s * nc + lin(p, x, y, z)] = p->bc_value[s][f];
                }

    /* Cahn-Hilliard: first Laplacian pass, mu = f'(c) - kappa Lap c with
     * f'(c) = 2 c (c - 1)(2 c - 1), over every cell of species 2 */
    if (p->model == ORC_CH_FRONT) {
        const double kappa = p->p[2];
        const double* c = cur + 2 * nc;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    double cc = c[lin(p, x, y, z)];
                    double fp = 2.0 * cc * (cc - 1.0) * (2.0 * cc - 1.0);
                    mu[lin(p, x, y, z)] = fp - kappa * laplacian(p, c, 2, x, y, z);
                }
    }
    /* Table 1, row 3: the bracket eps c - gamma c^3 + sigma Lap c over every
     * cell of species 2, then (below) -lambda Lap of it */
    if (p->model == ORC_CH_TABLE1) {
        const double eps = p->p[3], gamma = p->p[4], sigma = p->p[5];
        const double* c = cur + 2 * nc;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    double cc = c[lin(p, x, y, z)];
                    mu[lin(p, x, y, z)] = eps * cc - gamma * cc * cc * cc
                                        + sigma * laplacian(p, c, 2, x, y, z);
                }
    }

    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int64_t i = lin(p, x, y, z);
                double v[ORC_MAXS], r[ORC_MAXS];
                for (int s = 0; s < ns; ++s) v[s] = cur[s * nc + i];
                reaction(p, v, r);
                const double u = p->wind_kind == ORC_WIND_3D ? 0.0 : orc_wind(p, z);
                double u3[3] = {0.0, 0.0, 0.0};
                if (p->wind_kind == ORC_WIND_3D) wind3(p, (double)n * p->dt, u3);
                for (int s = 0; s < ns; ++s) {
                    const double* f = cur + s * nc;
                    double rate = r[s];
                    if (p->stencil == 19)
                        rate += p->D[s][0] * laplacian19(p, f, s, x, y, z);
                    else
                        for (int a = 0; a < 3; ++a)
                            rate += p->D[s][a] * second_diff(p, f, s, x, y, z, a);
                    if (p->wind_kind == ORC_WIND_3D)
                        for (int a = 0; a < 3; ++a) rate += upwind(p, f, s, x, y, z, a, u3[a]);
                    if (u != 0.0) {
                        /* first-order upwind: -u dc/dx from the upstream side */
                        if (u > 0.0)
                            rate -= u * (v[s] - nb(p, f, s, x, y, z, 0, -1)) / p->h;
                        else
                            rate -= u * (nb(p, f, s, x, y, z, 0, +1) - v[s]) / p->h;
                    }
                    if (p->model == ORC_CH_TABLE1 && s == 2)
                        rate -= p->p[2] * laplacian(p, mu, 2, x, y, z);
                    if (p->model == ORC_CH_FRONT && s == 2) {
                        /* second Laplacian pass: M Lap mu, mu taking the
                         * boundary rule of species 2 */
                        rate += p->p[1] * laplacian(p, mu, 2, x, y, z);
                    }
                    if (s == p->src_species && x == p->src_x && y == p->src_y
                        && z == p->src_z)
                        rate += p->src_rate;
                    double out = v[s] + p->dt * rate;
                    int hf = held_face(p, s, x, y, z);
                    if (hf >= 0) out = p->bc_value[s][hf];
                    nxt[s * nc + i] = out;
                }
            }
}

int orc_run(const orc_problem* p, double* state, int64_t nsteps)
{
    if (check(p) != 0 || !state || nsteps < 0) return -1;
    const int64_t nc = (int64_t)p->nx * p->ny * p->nz;
    double* other = (double*)malloc(sizeof(double) * nc * p->ns);
    double* mu = (double*)malloc(sizeof(double) * nc);
    if (!other || !mu) { free(other); free(mu); return -1; }
    double* cur = state;
    double* nxt = other;
    for (int64_t t = 0; t < nsteps; ++t) {
        step(p, cur, nxt, mu, p->n0 + t);
        double* tmp = cur; cur = nxt; nxt = tmp;
    }
    if (cur != state) memcpy(state, cur, sizeof(double) * nc * p->ns);
    free(other);
    free(mu);
    return 0;
}
