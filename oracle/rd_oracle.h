/*
 * rd_oracle.h -- plain FP64, single-threaded CPU reference stepper.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (the method of lines of Section 2 of the paper):
 *   eq. (1)  dc/dt = div(D grad c) + R(c), D diagonal (here per species and
 *            per axis), plus first-order upwind advection (Section 4.1,
 *            Table 1 row 4) and a point emission term E;
 *   7-point Laplacian per axis: (c[i-1] + c[i+1] - 2 c[i]) / h^2;
 *   eqs. (3)-(4) the 19-point Laplacian (stencil = 19): (1 / 6h^2) times
 *            the sum of T_pqr c[i+p, j+q, k+r] over the 3x3x3 block, with
 *            the weights of eq. (4) (-24 centre, 2 face, 1 edge, 0
 *            corner); one diffusivity per species (D[s][0..2] equal);
 *   eq. (5)  forward Euler: c(t+dt) = c(t) + dt * [diffusion + R + ...],
 *            every term taken from level t (the time-dependent wind of
 *            ORC_WIND_3D too, at t = n dt for step n = 0, 1, ...);
 *   Table 3  host loop: set boundary values, update all points from the
 *            "first" arrays into the "second" arrays, swap.
 *   Section 4.1 (Cahn-Hilliard): the biharmonic term is computed as a
 *            Laplacian, boundary conditions applied again, then a second
 *            Laplacian -- done here with a separate mu array, as two passes.
 *
 * Boundary kinds per species and face (-x,+x,-y,+y,-z,+z):
 *   ORC_NEUMANN   zero flux: the ghost value outside a face equals the
 *                 cell on the face;
 *   ORC_PERIODIC  wrap-around (both faces of an axis);
 *   ORC_DIRICHLET the outermost layer of cells on that face is a boundary
 *                 layer held at bc_value (set before each step, never
 *                 updated), as the paper stores boundary points in the
 *                 outermost grid layer (Section 4.1, boundary kernels).
 * The 19-point stencil also reads edge neighbours (two axes shifted); their
 * ghost index applies each crossed axis's rule in turn, as the paper's
 * separate edge kernels fill the edges from the faces (Section 4.1).
 */
#ifndef RD_ORACLE_H
#define RD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_NEUMANN = 0, ORC_PERIODIC = 1, ORC_DIRICHLET = 2 };
enum { ORC_DIFFUSION = 0, ORC_BRUSSELATOR = 1, ORC_CH_FRONT = 2, ORC_AIR = 3, ORC_TURING = 4,
       ORC_CH_TABLE1 = 5 };
enum { ORC_WIND_NONE = 0, ORC_WIND_LOG = 1, ORC_WIND_CONST = 2, ORC_WIND_3D = 3 };

#define ORC_MAXS 4

typedef struct orc_problem {
    int32_t nx, ny, nz, ns;
    int32_t model;
    int32_t wind_kind;
    double h, dt;
    double D[ORC_MAXS][3];           /* diffusivity per species, per axis   */
    int32_t bc[ORC_MAXS][6];
    double bc_value[ORC_MAXS][6];
    /* model constants:
     *   BRUSSELATOR  p[0]=a, p[1]=b
     *   CH_FRONT     p[0]=k (a+b->c), p[1]=M (mobility), p[2]=kappa
     *   AIR          p[0]=j (NO2 -> NO + O3), p[1]=k (NO + O3 -> NO2)
     *   TURING       p[0]=alpha, p[1]=beta, p[2]=gamma (Table 1, row 2)
     *   CH_TABLE1    p[0]=k1, p[1]=k2, p[2]=lambda, p[3]=eps, p[4]=gamma,
     *                p[5]=sigma (Table 1, row 3: c3 moves by
     *                -lambda Lap(eps c3 - gamma c3^3 + sigma Lap c3))     */
    double p[8];
    double wind_u0;                  /* scale of u_x                        */
    int32_t src_x, src_y, src_z, src_species;   /* src_species < 0: none    */
    double src_rate;
    int32_t stencil;                 /* 7 (or 0): 7-point; 19: eqs. (3)-(4) */
    int32_t pad0;
    /* ORC_WIND_3D (Table 1, row 4): u = (w3[0], w3[1], w3[2] sin(t / w3[3]))
     * with t the time at the start of the step, n dt; first-order upwind
     * along each axis                                                      */
    double w3[4];
    int64_t n0;                      /* index of the first step orc_run takes */
} orc_problem;

/* Advance ``state`` (ns x nz x ny x nx doubles, x fastest) by nsteps
 * forward-Euler steps, in place.  Returns 0, or -1 on a bad problem or
 * allocation failure. */
int orc_run(const orc_problem* p, double* state, int64_t nsteps);

/* Wind speed u_x at height index z (cells), as used by orc_run. */
double orc_wind(const orc_problem* p, int z);

#ifdef __cplusplus
}
#endif
#endif
