/*
 * FP64 CPU oracle for the coupled D3Q19 lattice Boltzmann time step of
 * Rettinger & Ruede, "A comparative study of fluid-particle coupling methods
 * for fully resolved lattice Boltzmann simulations" (arXiv:1702.04910).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header or
 * table with the CUDA library: the lattice table below is written out here
 * from the paper's D3Q19 convention on its own.
 *
 * Structure: the paper's algorithms in the paper's order.
 *   - PSM global step  = Algorithm 2 (Sec. 2.3): solid fractions, collision
 *     with Eq. (20), (26), force/torque Eq. (28)-(29), stream Eq. (2), rigid
 *     body update.
 *   - MEM global step  = Algorithm 1 (Sec. 2.2): per LBM subcycle collide
 *     Eq. (1) with TRT Eq. (9), boundary conditions Eq. (12) / (14) / (15),
 *     stream Eq. (2), link forces Eq. (16); then average, total force/torque
 *     Eq. (17)-(18), rigid body update, re-mapping and PDF reconstruction
 *     Eq. (19).
 * The stored state between global steps is the pre-collision PDF field f
 * (the state right after streaming).  The last post-collision field f~ is kept
 * as well, because the GPU library stores post-collision values.
 *
 * Every arithmetic step is written literally, in FP64, with no blocking,
 * fusion or reordering.  Build with -ffp-contract=off so that no fused
 * multiply-add changes rounding between machines.
 *
 * Readings of points the paper leaves open:
 *  R1  D3Q19 order: 0 rest; 1..6 axis (+x,-x,+y,-y,+z,-z); 7..18 diagonals
 *      in opposite pairs; weights 1/3, 1/18, 1/36 (Sec. 2.1 "as in Qian").
 *  R2  Forcing Eq. (7) is applied unsplit, without a (1 - 1/2tau) factor;
 *      f_eq and F_q use U, the output velocity is u of Eq. (8).
 *  R3  PSM fluid part: BGK as printed in Eq. (20), or TRT when requested.
 *  R4  rho in M1..M3 (Eq. 23-25) is the cell fluid density rho_f.
 *  R5  Cell centres sit at integer + 1/2.  PSM v_s and torque arm at the cell
 *      centre; MEM boundary point x_b = x + delta_q c_q (BB: delta_q = 1/2).
 *  R6  MEM: a cell is solid iff its centre is inside or on the sphere
 *      (|x_c - X_p| <= R), minimum image in periodic directions.
 *  R7  delta_q: smallest root t of |x + t c_q - X_p| = R, clamped to [0,1].
 *  R8  CLI needs f~_q(x - c_q); where x - c_q is not a fluid cell the link
 *      falls back to BB (delta = 1/2 weights, x_b still at delta_q).
 *  R9  Refilling velocity constraint (Sec. 2.2, "moment space"): add
 *      c_q . (rho0 v - j) / 10 to each f_q; sum_q c_qa^2 = 10 on D3Q19, so
 *      only the momentum moment of an orthogonal moment basis changes.
 * R10  q_n = argmax_q n . c_q over the unnormalised c_q, ties to the lowest q.
 * R11  Fewer fluid neighbours: 3 -> (3,-3,1), 2 -> (2,-1), 1 -> (1),
 *      0 -> f_eq(rho_bar, v), rho_bar = mean density of the usable fluid
 *      cells among the 18 neighbours (rho0 if none).  A usable neighbour is
 *      inside the domain and fluid under both the old and the new mapping.
 * R12  Rigid body: explicit Euler over the time the fluid advanced in the
 *      global step (dt = number of LBM subcycles): X += dt U; U += dt F/m;
 *      W += dt T/I; m = rho_p pi D^3/6, I = m D^2/10; total force
 *      F_hyd + (rho_p - rho0) V g.  X is wrapped into periodic directions.
 * R13  Wall contact (closed z walls, optional): the sphere surface is kept at
 *      least one cell from a wall and the wall-normal velocity towards it is
 *      zeroed.
 * R14  MEM subcycles use the particle state of the start of the global step;
 *      the reported force is the average of the subcycle forces.
 * R15  PSM solid fraction: uniform n^3 supersampling at (i + 1/2)/n inside
 *      the cell, a sample is inside iff |p - X_p| <= R (config: n = 4).
 * R16  Host-side particle replacement between steps (MEM): cells uncovered
 *      relative to the current mapping are set to f_eq(rho0, v).
 * R17  MEM MR, Eq. (15): the paper takes kappa, alpha and f^pc from tables of
 *      the cited TRT study, which are not at hand.  They are derived here
 *      from the second-order no-slip requirement instead: along the link the
 *      steady TRT recurrence (pre-collision non-equilibrium n^+- of the
 *      equilibrium parts e^+-, Lambda_+- = 1/lambda_+- - 1/2 in magnitude) is
 *      solved for equilibria quadratic in the link coordinate, and Eq. (15)
 *      is required to return the population that would arrive from x + c_q
 *      whenever u(x_b) = v(x_b), for any wall velocity, density, velocity
 *      slope, velocity curvature and pressure gradient along the link.
 *      With kappa_1 = 1, kappabar_-1 = -kappa_0 and kappabar_-2 = -kappa_-1
 *      (the pairing of Eq. (14)) the solution is unique:
 *        kappa_0 = (1 - 2 d - 2 d^2)/(1 + d)^2, kappa_-1 = d^2/(1 + d)^2,
 *        alpha = 4/(1 + d)^2,
 *        f^pc = -8 Lambda_- / ((2 Lambda_- + 1)(1 + d)^2) n^-_q(x, t),
 *      d = delta_q, n^-_q = odd part of f_q - f_eq,q of the PRE-collision
 *      populations at x (the stored old values of Sec. 4).  MR needs x - c_q
 *      and x - 2 c_q to be fluid; where only x - c_q is, the link uses
 *      Eq. (14) (CLI), else Eq. (12) with the BB weights (as R8).
 * R30  LBM subcycles with PSM: Algorithm 2 runs one sweep per step, but the
 *      settling benchmark of Sec. 4.1 states that two LBM subcycles are run
 *      and their forces averaged.  With subcycles = 2 a PSM step does both
 *      sweeps with the particle state of the start of the step (as R14),
 *      averages the forces and advances the particle by dt = 2.
 * R27  Open z boundaries of the benchmark frame (Sec. 4.1), bc_z = 2: at the
 *      bottom the velocity bounce-back of Eq. (12) with the inflow velocity
 *      u_in; at the top the outflow of Sec. 4.1, f_qbar(x,t+1) = -f~_q(x,t)
 *      + 2 f_eq,+_q(rho_out, u(x,t)), with f_eq,+ the even part of Eq. (3)
 *      and u(x,t) the velocity of Eq. (8) of the boundary cell before the
 *      stream.
 * R32  Re-mapping momentum (optional, remap_charge = 1; Algorithm 1 has no
 *      such step, so the default is 0).  The re-mapping at the end of a MEM
 *      step removes from the fluid the momentum sum_q c_q f_q of every cell
 *      the particle covers and creates that of every cell it uncovers (after
 *      the refill of Eq. (19)).  With the option on, the difference dP
 *      (created minus removed) and its moment dL about the particle's new
 *      centre (arm x_c - X_p) are kept, and the next step's averaged force
 *      and torque become F - dP/dt and T - dL/dt, dt the step's lattice time
 *      (the LBM subcycles), before the rigid-body update: the particle then
 *      gives or takes what the fluid gained or lost.  Replacing particles
 *      from the host clears the pending amounts.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NQ 19
static const double PI = 3.14159265358979323846;

/* ---- D3Q19 lattice (R1) ------------------------------------------------ */
static const int CQ[NQ][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const int OPP[NQ] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9,
                            12, 11, 14, 13, 16, 15, 18, 17};
static const double W0 = 1.0 / 3.0, W1 = 1.0 / 18.0, W2 = 1.0 / 36.0;
static double WQ[NQ];
static const double INV_CS2 = 3.0; /* 1/c_s^2 in lattice units (c_s^2 = 1/3) */

enum { ORC_PSM_M1B1 = 0, ORC_PSM_M2B2 = 1, ORC_PSM_M3B2 = 2,
       ORC_MEM_BB = 3, ORC_MEM_CLI = 4, ORC_MEM_MR = 5, ORC_NONE = 6 };
enum { ORC_BGK = 0, ORC_TRT = 1 };
enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_UNSTABLE = -4,
       ORC_ERR_DOMAIN = -5, ORC_ERR_UNSUPPORTED = -7 };

typedef struct {
    int nx, ny, nz;
    int bc_z;          /* 0 periodic in z, 1 resting no-slip walls at z=0, nz,
                          2 inflow at z=0 and outflow at z=nz (R27) */
    int collision;     /* ORC_BGK / ORC_TRT */
    int coupling;      /* ORC_PSM_* / ORC_MEM_* / ORC_NONE */
    double tau, magic; /* relaxation time, Lambda of Eq. (11) */
    double fext[3];    /* fluid force density f_ext, Eq. (7) */
    double gravity[3]; /* acceleration acting on particles */
    double rho0;
    int subsample;     /* n of the n^3 supersampling (R15) */
    int subcycles;     /* LBM sweeps per global step (MEM: 2) */
    int wall_contact;  /* R13 */
    double inflow[3];  /* bc_z = 2: inflow velocity at z = 0 (R27) */
    double rho_out;    /* bc_z = 2: outflow density at z = nz (R27) */
    int remap_charge;  /* MEM: charge the re-mapping momentum (R32) */
} orc_params;

typedef struct {
    double x[3], u[3], omega[3];
    double diameter, density;
    int fixed;
} orc_particle;

typedef struct {
    orc_params p;
    long n;              /* cells */
    double lam_p, lam_m; /* lambda_+ , lambda_- of Eq. (9) */
    double *f;           /* pre-collision PDFs, [q][z][y][x] */
    double *ft;          /* last post-collision PDFs */
    int np;
    orc_particle *part;
    int *solid;          /* MEM mapping: 0 fluid, s+1 inside particle s */
    int mapped;
    double *eps;         /* PSM: eps_s per cell, [s][cell] for current P */
    double *force, *torque; /* last hydrodynamic force / torque, [s][3] */
    double *fsum, *tsum;    /* per-subcycle accumulators */
    double *charge;         /* R32: momentum / angular momentum the last
                               re-mapping gave the fluid, [s][6] */
    long steps;
} orc_sim;

static void init_weights(void) {
    WQ[0] = W0;
    for (int q = 1; q <= 6; ++q) WQ[q] = W1;
    for (int q = 7; q < NQ; ++q) WQ[q] = W2;
}

/* ---- small helpers ------------------------------------------------------ */
static long cell_index(const orc_sim *s, int x, int y, int z) {
    return (long)x + (long)s->p.nx * ((long)y + (long)s->p.ny * (long)z);
}
static int wrap(int i, int n) { return ((i % n) + n) % n; }

/* Neighbour of (x,y,z) along integer offset (dx,dy,dz); returns -1 when the
 * neighbour lies beyond a closed z wall. */
static long neighbour(const orc_sim *s, int x, int y, int z, int dx, int dy, int dz) {
    int xx = wrap(x + dx, s->p.nx), yy = wrap(y + dy, s->p.ny), zz = z + dz;
    if (s->p.bc_z) {
        if (zz < 0 || zz >= s->p.nz) return -1;
    } else {
        zz = wrap(zz, s->p.nz);
    }
    return cell_index(s, xx, yy, zz);
}

/* Minimum-image separation a - b along one axis of length L (periodic). */
static double min_image(double d, double L, int periodic) {
    if (!periodic) return d;
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}
static void separation(const orc_sim *s, const double a[3], const double b[3], double d[3]) {
    d[0] = min_image(a[0] - b[0], (double)s->p.nx, 1);
    d[1] = min_image(a[1] - b[1], (double)s->p.ny, 1);
    d[2] = min_image(a[2] - b[2], (double)s->p.nz, !s->p.bc_z);
}
static void cross(const double a[3], const double b[3], double r[3]) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
static void cell_centre(int x, int y, int z, double c[3]) {
    c[0] = x + 0.5; c[1] = y + 0.5; c[2] = z + 0.5;
}
static int is_psm(int c) { return c == ORC_PSM_M1B1 || c == ORC_PSM_M2B2 || c == ORC_PSM_M3B2; }
static int is_mem(int c) { return c == ORC_MEM_BB || c == ORC_MEM_CLI || c == ORC_MEM_MR; }

/* ---- Eq. (3): incompressible equilibrium -------------------------------
 * With c_s^2 = 1/3: 1/c_s^2 = 3, 1/(2 c_s^4) = 9/2, 1/(2 c_s^2) = 3/2. */
double orc_feq(int q, double rho_f, const double U[3], double rho0) {
    double cu = CQ[q][0] * U[0] + CQ[q][1] * U[1] + CQ[q][2] * U[2];
    double uu = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    return WQ[q] * (rho_f + rho0 * (3.0 * cu + 4.5 * (cu * cu) - 1.5 * uu));
}

/* ---- Eq. (4): moments ---------------------------------------------------- */
static void moments(const double fc[NQ], double rho0, double *rho, double U[3]) {
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < NQ; ++q) {
        r += fc[q];
        for (int a = 0; a < 3; ++a) j[a] += fc[q] * CQ[q][a];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) U[a] = j[a] / rho0;
}

/* ---- Eq. (7): forcing term -----------------------------------------------
 * F_q = w_q [ (c_q - U)/c_s^2 + (c_q . U) c_q / c_s^4 ] . f_ext, with
 * 1/c_s^2 = 3 and 1/c_s^4 = 9. */
static double forcing(int q, const double U[3], const double fext[3]) {
    double cu = CQ[q][0] * U[0] + CQ[q][1] * U[1] + CQ[q][2] * U[2];
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
        s += (3.0 * (CQ[q][a] - U[a]) + 9.0 * cu * CQ[q][a]) * fext[a];
    return WQ[q] * s;
}

/* ---- Eq. (5) BGK and Eq. (9)-(10) TRT fluid collision operators ---------- */
static void fluid_collision(const orc_sim *s, const double fc[NQ], double rho,
                            const double U[3], double C[NQ]) {
    double feq[NQ];
    for (int q = 0; q < NQ; ++q) feq[q] = orc_feq(q, rho, U, s->p.rho0);
    if (s->p.collision == ORC_BGK) {
        for (int q = 0; q < NQ; ++q) C[q] = (feq[q] - fc[q]) / s->p.tau;
    } else {
        for (int q = 0; q < NQ; ++q) {
            int qb = OPP[q];
            double fp = 0.5 * (fc[q] + fc[qb]), fm = 0.5 * (fc[q] - fc[qb]);
            double ep = 0.5 * (feq[q] + feq[qb]), em = 0.5 * (feq[q] - feq[qb]);
            C[q] = s->lam_p * (fp - ep) + s->lam_m * (fm - em);
        }
    }
}

/* ---- Eq. (13): rigid-body velocity at a point ---------------------------- */
static void body_velocity(const orc_sim *s, const orc_particle *P, const double x[3], double v[3]) {
    double r[3], wxr[3];
    separation(s, x, P->x, r);
    cross(P->omega, r, wxr);
    for (int a = 0; a < 3; ++a) v[a] = P->u[a] + wxr[a];
}

/* R6: is point x inside (or on) particle P */
static int point_inside(const orc_sim *s, const orc_particle *P, const double x[3]) {
    double d[3];
    separation(s, x, P->x, d);
    double R = 0.5 * P->diameter;
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= R * R;
}

/* ---- PSM solid fraction by supersampling (Sec. 2.3, R15) ----------------- */
static double solid_fraction(const orc_sim *s, const orc_particle *P, int x, int y, int z) {
    int n = s->p.subsample, inside = 0;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double pt[3] = {x + (i + 0.5) / n, y + (j + 0.5) / n, z + (k + 0.5) / n};
                inside += point_inside(s, P, pt);
            }
    return (double)inside / ((double)n * n * n);
}

/* Cells of the axis-aligned box around particle P (used to skip cells that
 * cannot intersect it; the box is one cell wider than the sphere). */
static void particle_box(const orc_sim *s, const orc_particle *P, int lo[3], int hi[3]) {
    double R = 0.5 * P->diameter;
    int nn[3] = {s->p.nx, s->p.ny, s->p.nz};
    for (int a = 0; a < 3; ++a) {
        lo[a] = (int)floor(P->x[a] - R) - 1;
        hi[a] = (int)floor(P->x[a] + R) + 1;
        if ((a == 2 && s->p.bc_z) || hi[a] - lo[a] + 1 > nn[a]) {
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > nn[a] - 1) hi[a] = nn[a] - 1;
        }
    }
}

static void compute_solid_fractions(orc_sim *s) {
    memset(s->eps, 0, sizeof(double) * (size_t)s->np * (size_t)s->n);
    for (int p = 0; p < s->np; ++p) {
        int lo[3], hi[3];
        particle_box(s, &s->part[p], lo, hi);
#pragma omp parallel for schedule(dynamic)
        for (int z = lo[2]; z <= hi[2]; ++z)
            for (int y = lo[1]; y <= hi[1]; ++y)
                for (int x = lo[0]; x <= hi[0]; ++x) {
                    int xx = wrap(x, s->p.nx), yy = wrap(y, s->p.ny);
                    int zz = s->p.bc_z ? z : wrap(z, s->p.nz);
                    s->eps[(size_t)p * s->n + cell_index(s, xx, yy, zz)] =
                        solid_fraction(s, &s->part[p], xx, yy, zz);
                }
    }
}

/* ---- MEM binary mapping (R6) --------------------------------------------- */
static void map_particles(const orc_sim *s, int *solid) {
#pragma omp parallel for
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                double c[3];
                cell_centre(x, y, z, c);
                int owner = 0;
                for (int p = 0; p < s->np && !owner; ++p)
                    if (point_inside(s, &s->part[p], c)) owner = p + 1;
                solid[cell_index(s, x, y, z)] = owner;
            }
}

/* ---- Stream, Eq. (2), with resting halfway bounce-back at closed z walls --
 * Pushes f~ of every non-solid cell to its neighbours.  Links that end in a
 * MEM solid cell are left for the boundary condition. */
static void stream(orc_sim *s) {
    int mem = is_mem(s->p.coupling);
    const int nxy = s->p.nx * s->p.ny;
    double *uout = NULL;
    if (s->p.bc_z == 2) {
        /* R27: Eq. (8) velocity of the top-plane cells at time t, taken
         * before the stream overwrites f */
        uout = (double *)malloc(sizeof(double) * 3 * (size_t)nxy);
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = cell_index(s, x, y, s->p.nz - 1);
                double fc[NQ], rho, U[3];
                for (int q = 0; q < NQ; ++q) fc[q] = s->f[(long)q * s->n + i];
                moments(fc, s->p.rho0, &rho, U);
                for (int a = 0; a < 3; ++a)
                    uout[3 * (x + s->p.nx * y) + a] = U[a] + s->p.fext[a] / (2.0 * s->p.rho0);
            }
    }
#pragma omp parallel for
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (mem && s->solid[i]) continue;
                for (int q = 0; q < NQ; ++q) {
                    long j = neighbour(s, x, y, z, CQ[q][0], CQ[q][1], CQ[q][2]);
                    if (j < 0) {
                        double v = s->ft[(long)q * s->n + i];
                        if (s->p.bc_z == 2 && CQ[q][2] < 0) {
                            /* inflow: velocity bounce-back, Eq. (12) with u_in */
                            double cu = 0.0;
                            for (int a = 0; a < 3; ++a) cu += CQ[q][a] * s->p.inflow[a];
                            v = v - 2.0 * WQ[q] * s->p.rho0 * cu * INV_CS2;
                        } else if (s->p.bc_z == 2) {
                            /* outflow (R27) */
                            const double *u = &uout[3 * (x + s->p.nx * y)];
                            double cu = 0.0, uu = 0.0;
                            for (int a = 0; a < 3; ++a) {
                                cu += CQ[q][a] * u[a];
                                uu += u[a] * u[a];
                            }
                            double feq_even = WQ[q] * (s->p.rho_out +
                                                       s->p.rho0 * (0.5 * INV_CS2 * INV_CS2 * cu * cu -
                                                                    0.5 * INV_CS2 * uu));
                            v = -v + 2.0 * feq_even;
                        }
                        s->f[(long)OPP[q] * s->n + i] = v;
                    } else if (mem && s->solid[j]) {
                        /* handled by mem_boundary() */
                    } else {
                        s->f[(long)q * s->n + j] = s->ft[(long)q * s->n + i];
                    }
                }
            }
    free(uout);
}

/* Force/torque partials are kept per z plane so that the sum order does not
 * depend on how many threads run the plane loop; planes are added in z order. */
static void sum_planes(const orc_sim *s, const double *Fz, const double *Tz, double *F, double *T) {
    size_t np3 = 3 * (size_t)s->np;
    for (int z = 0; z < s->p.nz; ++z)
        for (size_t k = 0; k < np3; ++k) {
            F[k] += Fz[(size_t)z * np3 + k];
            T[k] += Tz[(size_t)z * np3 + k];
        }
}

/* ---- MEM link geometry ---------------------------------------------------- */
/* R7: fraction delta_q of the link x -> x + c_q where the sphere surface is. */
static double link_delta(const orc_sim *s, const orc_particle *P, const double x[3], int q) {
    double d[3];
    separation(s, x, P->x, d);
    double R = 0.5 * P->diameter;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = 0; k < 3; ++k) {
        a += (double)(CQ[q][k] * CQ[q][k]);
        b += d[k] * CQ[q][k];
        c += d[k] * d[k];
    }
    c -= R * R;
    double disc = b * b - a * c;
    if (disc < 0.0) disc = 0.0;
    double t = (-b - sqrt(disc)) / a;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    return t;
}

/* delta used by the active boundary scheme: BB -> 1/2, CLI -> R7 */
static double scheme_delta(const orc_sim *s, const orc_particle *P, const double x[3], int q) {
    if (s->p.coupling == ORC_MEM_BB) return 0.5;
    return link_delta(s, P, x, q);
}

/* Eq. (15) with the coefficients of R17.  q is the link direction (towards
 * the wall), qbar its opposite; ft_q0/1/2 = f~_q at x, x - c_q, x - 2 c_q;
 * ft_qb0/1 = f~_qbar at x, x - c_q; n_minus = n^-_q(x, t) (R17); e_wall =
 * w_q rho0 v(x_b) . c_q / c_s^2; Lambda_m = 1/|lambda_-| - 1/2. */
double orc_mr_link(double delta, double Lambda_m, double ft_q0, double ft_q1, double ft_q2,
                   double ft_qb0, double ft_qb1, double n_minus, double e_wall) {
    double d1 = (1.0 + delta) * (1.0 + delta);
    double kappa1 = 1.0;
    double kappa0 = (1.0 - 2.0 * delta - 2.0 * delta * delta) / d1;
    double kappam1 = delta * delta / d1;
    double kappabm1 = -kappa0;
    double kappabm2 = -kappam1;
    double alpha = 4.0 / d1;
    double kpc = -8.0 * Lambda_m / ((2.0 * Lambda_m + 1.0) * d1);
    double fpc = kpc * n_minus;
    return kappa1 * ft_q0 + kappa0 * ft_q1 + kappam1 * ft_q2 + kappabm1 * ft_qb0 +
           kappabm2 * ft_qb1 - alpha * e_wall + fpc;
}

/* Boundary value f_qbar(x, t+1) for fluid x whose neighbour x + c_q is solid:
 * Eq. (12) BB, Eq. (14) CLI or Eq. (15) MR.  fpre: pre-collision f(x, t). */
static double link_value(const orc_sim *s, int x, int y, int z, int q, const orc_particle *P,
                         const double fpre[NQ]) {
    long i = cell_index(s, x, y, z);
    int qb = OPP[q];
    double xc[3], xb[3], v[3];
    cell_centre(x, y, z, xc);
    double delta = scheme_delta(s, P, xc, q);
    for (int a = 0; a < 3; ++a) xb[a] = xc[a] + delta * CQ[q][a];
    body_velocity(s, P, xb, v);
    double vc = v[0] * CQ[q][0] + v[1] * CQ[q][1] + v[2] * CQ[q][2];
    double ftq = s->ft[(long)q * s->n + i];
    double e_wall = (WQ[q] * INV_CS2) * s->p.rho0 * vc;
    if (s->p.coupling == ORC_MEM_MR) {
        long jb = neighbour(s, x, y, z, -CQ[q][0], -CQ[q][1], -CQ[q][2]);
        long jb2 = neighbour(s, x, y, z, -2 * CQ[q][0], -2 * CQ[q][1], -2 * CQ[q][2]);
        if (jb >= 0 && !s->solid[jb] && jb2 >= 0 && !s->solid[jb2]) {
            /* n^-_q(x, t): odd part of the pre-collision non-equilibrium */
            double rho, U[3];
            moments(fpre, s->p.rho0, &rho, U);
            double n_minus = 0.5 * (fpre[q] - fpre[qb]) -
                             0.5 * (orc_feq(q, rho, U, s->p.rho0) - orc_feq(qb, rho, U, s->p.rho0));
            double Lambda_m = -1.0 / s->lam_m - 0.5;
            return orc_mr_link(delta, Lambda_m, ftq, s->ft[(long)q * s->n + jb],
                               s->ft[(long)q * s->n + jb2], s->ft[(long)qb * s->n + i],
                               s->ft[(long)qb * s->n + jb], n_minus, e_wall);
        }
        /* R17: x - 2 c_q missing, the CLI of Eq. (14) below (or BB) */
    }
    if (s->p.coupling == ORC_MEM_CLI || s->p.coupling == ORC_MEM_MR) {
        long jb = neighbour(s, x, y, z, -CQ[q][0], -CQ[q][1], -CQ[q][2]);
        if (jb >= 0 && !s->solid[jb]) {
            double kappa0 = (1.0 - 2.0 * delta) / (1.0 + 2.0 * delta);
            double alpha = 4.0 / (1.0 + 2.0 * delta);
            return ftq + kappa0 * s->ft[(long)q * s->n + jb] -
                   kappa0 * s->ft[(long)qb * s->n + i] -
                   alpha * e_wall;
        }
        /* R8: second node missing, fall back to the BB weights */
    }
    return ftq - 2.0 * e_wall;
}

/* "Apply boundary conditions", Algorithm 1: Eq. (12) / (14) / (15) on every
 * fluid-solid link.  Writes the post-stream value f_qbar(x, t+1); the values
 * of one cell are all computed before any is written, because MR reads the
 * cell's pre-collision populations f(x, t). */
static void mem_boundary(orc_sim *s) {
#pragma omp parallel for
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (s->solid[i]) continue;
                double fpre[NQ], val[NQ];
                int set[NQ];
                for (int q = 0; q < NQ; ++q) {
                    fpre[q] = s->f[(long)q * s->n + i];
                    set[q] = 0;
                }
                for (int q = 1; q < NQ; ++q) {
                    long j = neighbour(s, x, y, z, CQ[q][0], CQ[q][1], CQ[q][2]);
                    if (j < 0 || !s->solid[j]) continue;
                    const orc_particle *P = &s->part[s->solid[j] - 1];
                    val[q] = link_value(s, x, y, z, q, P, fpre);
                    set[q] = 1;
                }
                for (int q = 1; q < NQ; ++q)
                    if (set[q]) s->f[(long)OPP[q] * s->n + i] = val[q];
            }
}

/* "Calculate hydrodynamic forces", Algorithm 1: Eq. (16), summed per
 * particle with the torque arm x_b - X_p, Eq. (17)-(18). */
static void mem_link_forces(orc_sim *s, double *Fout, double *Tout) {
    size_t np3 = 3 * (size_t)s->np;
    double *Fz = (double *)calloc((size_t)s->p.nz * np3 + 1, sizeof(double));
    double *Tz = (double *)calloc((size_t)s->p.nz * np3 + 1, sizeof(double));
#pragma omp parallel for
    for (int z = 0; z < s->p.nz; ++z) {
        double *F = Fz + (size_t)z * np3, *T = Tz + (size_t)z * np3;
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (s->solid[i]) continue;
                for (int q = 1; q < NQ; ++q) {
                    long j = neighbour(s, x, y, z, CQ[q][0], CQ[q][1], CQ[q][2]);
                    if (j < 0 || !s->solid[j]) continue;
                    int p = s->solid[j] - 1;
                    const orc_particle *P = &s->part[p];
                    int qb = OPP[q];
                    double xc[3], xb[3], v[3], arm[3], Fl[3], Tl[3];
                    cell_centre(x, y, z, xc);
                    double delta = scheme_delta(s, P, xc, q);
                    for (int a = 0; a < 3; ++a) xb[a] = xc[a] + delta * CQ[q][a];
                    body_velocity(s, P, xb, v);
                    double ftq = s->ft[(long)q * s->n + i];
                    double fqb = s->f[(long)qb * s->n + i];
                    for (int a = 0; a < 3; ++a)
                        Fl[a] = (CQ[q][a] - v[a]) * ftq - (CQ[qb][a] - v[a]) * fqb;
                    separation(s, xb, P->x, arm);
                    cross(arm, Fl, Tl);
                    for (int a = 0; a < 3; ++a) {
                        F[3 * p + a] += Fl[a];
                        T[3 * p + a] += Tl[a];
                    }
                }
            }
    }
    sum_planes(s, Fz, Tz, Fout, Tout);
    free(Fz);
    free(Tz);
}

/* Plain fluid collision Eq. (1) for every non-solid cell: f~ = f + C + F. */
static void collide_fluid(orc_sim *s) {
    int mem = is_mem(s->p.coupling);
#pragma omp parallel for
    for (long i = 0; i < s->n; ++i) {
        if (mem && s->solid[i]) continue;
        double fc[NQ], C[NQ], rho, U[3];
        for (int q = 0; q < NQ; ++q) fc[q] = s->f[(long)q * s->n + i];
        moments(fc, s->p.rho0, &rho, U);
        fluid_collision(s, fc, rho, U, C);
        for (int q = 0; q < NQ; ++q)
            s->ft[(long)q * s->n + i] = fc[q] + C[q] + forcing(q, U, s->p.fext);
    }
}

/* ---- PSM collision Eq. (20)-(26) with force/torque Eq. (28)-(29) -------- */
static void collide_psm(orc_sim *s, double *Fout, double *Tout) {
    double tau = s->p.tau;
    int M = s->p.coupling; /* M1B1, M2B2, M3B2 */
    size_t np3 = 3 * (size_t)s->np;
    double *Fz = (double *)calloc((size_t)s->p.nz * np3 + 1, sizeof(double));
    double *Tz = (double *)calloc((size_t)s->p.nz * np3 + 1, sizeof(double));
#pragma omp parallel for
    for (int z = 0; z < s->p.nz; ++z) {
        double *F = Fz + (size_t)z * np3, *T = Tz + (size_t)z * np3;
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = cell_index(s, x, y, z);
                double fc[NQ], Cf[NQ], feqU[NQ], rho, U[3], xc[3];
                for (int q = 0; q < NQ; ++q) fc[q] = s->f[(long)q * s->n + i];
                moments(fc, s->p.rho0, &rho, U);
                fluid_collision(s, fc, rho, U, Cf);
                for (int q = 0; q < NQ; ++q) feqU[q] = orc_feq(q, rho, U, s->p.rho0);
                cell_centre(x, y, z, xc);
                double B = 0.0, solid_sum[NQ];
                for (int q = 0; q < NQ; ++q) solid_sum[q] = 0.0;
                for (int p = 0; p < s->np; ++p) {
                    double e = s->eps[(size_t)p * s->n + i];
                    if (e <= 0.0) continue;
                    double Bs;
                    if (M == ORC_PSM_M1B1) Bs = e;                                   /* Eq. (21) */
                    else Bs = e * (tau - 0.5) / ((1.0 - e) + (tau - 0.5));          /* Eq. (22) */
                    B += Bs;
                    double vs[3], feqV[NQ], Cs[NQ];
                    body_velocity(s, &s->part[p], xc, vs);
                    for (int q = 0; q < NQ; ++q) feqV[q] = orc_feq(q, rho, vs, s->p.rho0);
                    for (int q = 0; q < NQ; ++q) {
                        int qb = OPP[q];
                        if (M == ORC_PSM_M1B1)                                         /* Eq. (23) */
                            Cs[q] = (fc[qb] - feqU[qb]) - (fc[q] - feqV[q]);
                        else if (M == ORC_PSM_M2B2)                                    /* Eq. (24) */
                            Cs[q] = (feqV[q] - fc[q]) + (1.0 - 1.0 / tau) * (fc[q] - feqU[q]);
                        else                                                           /* Eq. (25) */
                            Cs[q] = (fc[qb] - feqV[qb]) - (fc[q] - feqV[q]);
                    }
                    double Fs[3] = {0.0, 0.0, 0.0}, arm[3], Ts[3];
                    for (int q = 0; q < NQ; ++q) {
                        solid_sum[q] += Bs * Cs[q];
                        for (int a = 0; a < 3; ++a) Fs[a] += Cs[q] * CQ[OPP[q]][a];
                    }
                    for (int a = 0; a < 3; ++a) Fs[a] = Bs * Fs[a];
                    separation(s, xc, s->part[p].x, arm);
                    cross(arm, Fs, Ts);
                    for (int a = 0; a < 3; ++a) {
                        F[3 * p + a] += Fs[a];
                        T[3 * p + a] += Ts[a];
                    }
                }
                for (int q = 0; q < NQ; ++q)
                    s->ft[(long)q * s->n + i] = fc[q] + ((1.0 - B) * Cf[q] + solid_sum[q]) +
                                                (1.0 - B) * forcing(q, U, s->p.fext);
            }
    }
    sum_planes(s, Fz, Tz, Fout, Tout);
    free(Fz);
    free(Tz);
}

/* ---- rigid body update (R12, R13) ----------------------------------------- */
static int rigid_body_update(orc_sim *s, double dt) {
    int status = ORC_OK;
    for (int p = 0; p < s->np; ++p) {
        orc_particle *P = &s->part[p];
        if (P->fixed) continue;
        double D = P->diameter, R = 0.5 * D;
        double V = PI * D * D * D / 6.0;
        double m = P->density * V, I = m * D * D / 10.0;
        double Ft[3];
        for (int a = 0; a < 3; ++a)
            Ft[a] = s->force[3 * p + a] + (P->density - s->p.rho0) * V * s->p.gravity[a];
        for (int a = 0; a < 3; ++a) P->x[a] += dt * P->u[a];
        for (int a = 0; a < 3; ++a) P->u[a] += dt * Ft[a] / m;
        for (int a = 0; a < 3; ++a) P->omega[a] += dt * s->torque[3 * p + a] / I;
        double L[3] = {(double)s->p.nx, (double)s->p.ny, (double)s->p.nz};
        for (int a = 0; a < 3; ++a) {
            if (a == 2 && s->p.bc_z) continue;
            if (P->x[a] < 0.0) P->x[a] += L[a];
            else if (P->x[a] >= L[a]) P->x[a] -= L[a];
        }
        if (s->p.bc_z) {
            if (s->p.wall_contact) {
                if (P->x[2] - R < 1.0) { P->x[2] = R + 1.0; if (P->u[2] < 0.0) P->u[2] = 0.0; }
                if (P->x[2] + R > L[2] - 1.0) { P->x[2] = L[2] - 1.0 - R; if (P->u[2] > 0.0) P->u[2] = 0.0; }
            } else if (P->x[2] - R < 0.0 || P->x[2] + R > L[2]) {
                status = ORC_ERR_DOMAIN;
            }
        }
    }
    return status;
}

/* ---- MEM re-mapping and PDF reconstruction, Eq. (19), R9-R11 ------------ */
/* Adds sign * (j, (x_c - X_p) x j) of cell (x, y, z) with momentum
 * j = sum_q c_q f_q to particle P's six entries of `charge` (R32). */
static void add_cell_momentum(const orc_sim *s, const orc_particle *P, int x, int y, int z,
                              const double fc[NQ], double sign, double *charge) {
    double xc[3], arm[3], j[3] = {0.0, 0.0, 0.0}, L[3];
    for (int q = 0; q < NQ; ++q)
        for (int a = 0; a < 3; ++a) j[a] += CQ[q][a] * fc[q];
    cell_centre(x, y, z, xc);
    separation(s, xc, P->x, arm);
    cross(arm, j, L);
    for (int a = 0; a < 3; ++a) {
        charge[a] += sign * j[a];
        charge[3 + a] += sign * L[a];
    }
}

/* Re-mapping with the particle state in s->part and refilling of uncovered
 * cells (Sec. 2.2).  charge != NULL: also the R32 amounts, [s][6]. */
static void remap_and_refill(orc_sim *s, int use_extrapolation, double *charge) {
    int *old = s->solid;
    int *neu = (int *)malloc(sizeof(int) * (size_t)s->n);
    map_particles(s, neu);
    double rho0 = s->p.rho0;
    if (charge) {
        for (int k = 0; k < 6 * s->np; ++k) charge[k] = 0.0;
        /* covered cells lose their fluid momentum (pre-collision PDFs) */
        for (int z = 0; z < s->p.nz; ++z)
            for (int y = 0; y < s->p.ny; ++y)
                for (int x = 0; x < s->p.nx; ++x) {
                    long i = cell_index(s, x, y, z);
                    if (old[i] || !neu[i]) continue;
                    double fc[NQ];
                    for (int q = 0; q < NQ; ++q) fc[q] = s->f[(long)q * s->n + i];
                    add_cell_momentum(s, &s->part[neu[i] - 1], x, y, z, fc, -1.0,
                                      charge + 6 * (neu[i] - 1));
                }
    }
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = cell_index(s, x, y, z);
                if (!(old[i] && !neu[i])) continue;
                const orc_particle *P = &s->part[old[i] - 1];
                double xc[3], nrm[3], v[3], fnew[NQ];
                cell_centre(x, y, z, xc);
                body_velocity(s, P, xc, v);
                /* approximate normal direction q_n (R10) */
                separation(s, xc, P->x, nrm);
                double len = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
                if (len > 0.0) for (int a = 0; a < 3; ++a) nrm[a] /= len;
                int qn = 1;
                double best = -1e300;
                for (int q = 1; q < NQ; ++q) {
                    double d = nrm[0] * CQ[q][0] + nrm[1] * CQ[q][1] + nrm[2] * CQ[q][2];
                    if (d > best) { best = d; qn = q; }
                }
                /* consecutive usable fluid cells along c_qn (R11) */
                long nb[3];
                int m = 0;
                if (use_extrapolation) {
                    for (int k = 1; k <= 3; ++k) {
                        long j = neighbour(s, x, y, z, k * CQ[qn][0], k * CQ[qn][1], k * CQ[qn][2]);
                        if (j < 0 || old[j] || neu[j]) break;
                        nb[m++] = j;
                    }
                }
                if (m > 0) {
                    for (int q = 0; q < NQ; ++q) {
                        double f1 = s->f[(long)q * s->n + nb[0]];
                        if (m == 3)
                            fnew[q] = 3.0 * f1 - 3.0 * s->f[(long)q * s->n + nb[1]] +
                                      s->f[(long)q * s->n + nb[2]];
                        else if (m == 2)
                            fnew[q] = 2.0 * f1 - s->f[(long)q * s->n + nb[1]];
                        else
                            fnew[q] = f1;
                    }
                    /* velocity constraint in moment space (R9) */
                    double j[3] = {0.0, 0.0, 0.0};
                    for (int q = 0; q < NQ; ++q)
                        for (int a = 0; a < 3; ++a) j[a] += fnew[q] * CQ[q][a];
                    double dj[3];
                    for (int a = 0; a < 3; ++a) dj[a] = rho0 * v[a] - j[a];
                    for (int q = 0; q < NQ; ++q)
                        fnew[q] += (CQ[q][0] * dj[0] + CQ[q][1] * dj[1] + CQ[q][2] * dj[2]) / 10.0;
                } else {
                    double rbar = rho0;
                    if (use_extrapolation) {
                        double sum = 0.0;
                        int cnt = 0;
                        for (int q = 1; q < NQ; ++q) {
                            long j = neighbour(s, x, y, z, CQ[q][0], CQ[q][1], CQ[q][2]);
                            if (j < 0 || old[j] || neu[j]) continue;
                            double r = 0.0;
                            for (int k = 0; k < NQ; ++k) r += s->f[(long)k * s->n + j];
                            sum += r;
                            ++cnt;
                        }
                        if (cnt > 0) rbar = sum / cnt;
                    }
                    for (int q = 0; q < NQ; ++q) fnew[q] = orc_feq(q, rbar, v, rho0);
                }
                for (int q = 0; q < NQ; ++q) s->f[(long)q * s->n + i] = fnew[q];
                if (charge) add_cell_momentum(s, P, x, y, z, fnew, 1.0, charge + 6 * (old[i] - 1));
            }
    memcpy(s->solid, neu, sizeof(int) * (size_t)s->n);
    free(neu);
}

/* ---- public interface ------------------------------------------------------ */
orc_sim *orc_create(const orc_params *p) {
    init_weights();
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || !(p->tau > 0.5)) return NULL;
    if (p->coupling < 0 || p->coupling > ORC_NONE) return NULL;
    if (p->bc_z < 0 || p->bc_z > 2 || (p->bc_z == 2 && p->nz < 2)) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    if (s->p.subsample <= 0) s->p.subsample = 4;
    if (s->p.subcycles <= 0) s->p.subcycles = is_mem(p->coupling) ? 2 : 1;
    s->n = (long)p->nx * p->ny * p->nz;
    s->lam_p = -1.0 / p->tau;
    /* Eq. (11): (1/2 + 1/lambda_+)(1/2 + 1/lambda_-) = Lambda */
    if (p->collision == ORC_TRT)
        s->lam_m = 1.0 / (p->magic / (0.5 + 1.0 / s->lam_p) - 0.5);
    else
        s->lam_m = s->lam_p;
    s->f = (double *)calloc((size_t)NQ * s->n, sizeof(double));
    s->ft = (double *)calloc((size_t)NQ * s->n, sizeof(double));
    s->solid = (int *)calloc((size_t)s->n, sizeof(int));
    if (!s->f || !s->ft || !s->solid) { free(s->f); free(s->ft); free(s->solid); free(s); return NULL; }
    return s;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free(s->f); free(s->ft); free(s->solid); free(s->part); free(s->eps);
    free(s->force); free(s->torque); free(s->fsum); free(s->tsum); free(s->charge);
    free(s);
}

double orc_lambda_minus(const orc_sim *s) { return s->lam_m; }

void orc_lattice(int *c, double *w, int *opp) {
    init_weights();
    for (int q = 0; q < NQ; ++q) {
        for (int a = 0; a < 3; ++a) c[3 * q + a] = CQ[q][a];
        w[q] = WQ[q];
        opp[q] = OPP[q];
    }
}

int orc_set_particles(orc_sim *s, int np, const orc_particle *parts) {
    if (np < 0) return ORC_ERR_ARG;
    int remap = s->mapped && is_mem(s->p.coupling);
    if (np != s->np) {
        if (remap) return ORC_ERR_ARG; /* particle count is fixed once mapped */
        free(s->part); free(s->eps); free(s->force); free(s->torque); free(s->fsum); free(s->tsum);
        free(s->charge);
        s->np = np;
        s->part = (orc_particle *)calloc((size_t)(np > 0 ? np : 1), sizeof(orc_particle));
        s->eps = (double *)calloc((size_t)(np > 0 ? np : 1) * (size_t)s->n, sizeof(double));
        s->force = (double *)calloc((size_t)(3 * (np > 0 ? np : 1)), sizeof(double));
        s->torque = (double *)calloc((size_t)(3 * (np > 0 ? np : 1)), sizeof(double));
        s->fsum = (double *)calloc((size_t)(3 * (np > 0 ? np : 1)), sizeof(double));
        s->tsum = (double *)calloc((size_t)(3 * (np > 0 ? np : 1)), sizeof(double));
        s->charge = (double *)calloc((size_t)(6 * (np > 0 ? np : 1)), sizeof(double));
    }
    for (int k = 0; k < 6 * np; ++k) s->charge[k] = 0.0; /* R32 */
    if (np) memcpy(s->part, parts, sizeof(orc_particle) * (size_t)np);
    if (is_mem(s->p.coupling)) {
        if (remap) remap_and_refill(s, 0, NULL); /* R16 */
        else map_particles(s, s->solid);
        s->mapped = 1;
    }
    if (is_psm(s->p.coupling)) compute_solid_fractions(s);
    return ORC_OK;
}

/* Re-mapping and PDF reconstruction of Sec. 2.2 on its own, for the pins:
 * the particles take the given state (as after a rigid-body update) and
 * every cell they uncover is rebuilt from the current pre-collision field by
 * the same routine the MEM global step calls after its rigid-body update. */
/* MEM test hook: give the mapped particles a new state and run the
 * re-mapping and refill of Sec. 2.2 alone; the R32 amounts of that
 * re-mapping become the pending charge. */
int orc_move_and_refill(orc_sim *s, int np, const orc_particle *parts) {
    if (!is_mem(s->p.coupling) || !s->mapped || np != s->np) return ORC_ERR_ARG;
    if (np) memcpy(s->part, parts, sizeof(orc_particle) * (size_t)np);
    remap_and_refill(s, 1, s->charge);
    return ORC_OK;
}
void orc_get_charge(const orc_sim *s, double *out) {
    if (s->np > 0) memcpy(out, s->charge, sizeof(double) * 6 * (size_t)s->np);
}

int orc_get_particles(const orc_sim *s, orc_particle *out) {
    if (s->np) memcpy(out, s->part, sizeof(orc_particle) * (size_t)s->np);
    return s->np;
}

/* Pre-collision state at t = 0 set to f_eq(rho, u) everywhere. */
void orc_init_equilibrium(orc_sim *s, double rho, const double u[3]) {
    for (long i = 0; i < s->n; ++i)
        for (int q = 0; q < NQ; ++q) {
            double v = orc_feq(q, rho, u, s->p.rho0);
            s->f[(long)q * s->n + i] = v;
            s->ft[(long)q * s->n + i] = v;
        }
}

void orc_set_pdf(orc_sim *s, const double *f_pre) {
    memcpy(s->f, f_pre, sizeof(double) * (size_t)NQ * (size_t)s->n);
    memcpy(s->ft, f_pre, sizeof(double) * (size_t)NQ * (size_t)s->n);
}

/* which: 0 = current pre-collision f, 1 = last post-collision f~,
 *        2 = post-collision value the current f would have after a plain
 *            fluid collision Eq. (1) (used to compare MEM states). */
void orc_get_pdf(const orc_sim *s, int which, double *out) {
    if (which == 0) { memcpy(out, s->f, sizeof(double) * (size_t)NQ * s->n); return; }
    if (which == 1) { memcpy(out, s->ft, sizeof(double) * (size_t)NQ * s->n); return; }
#pragma omp parallel for
    for (long i = 0; i < s->n; ++i) {
        double fc[NQ], C[NQ], rho, U[3];
        for (int q = 0; q < NQ; ++q) fc[q] = s->f[(long)q * s->n + i];
        moments(fc, s->p.rho0, &rho, U);
        fluid_collision(s, fc, rho, U, C);
        for (int q = 0; q < NQ; ++q) out[(long)q * s->n + i] = fc[q] + C[q] + forcing(q, U, s->p.fext);
    }
}

void orc_get_forces(const orc_sim *s, double *F, double *T) {
    if (s->np == 0) return;
    memcpy(F, s->force, sizeof(double) * 3 * (size_t)s->np);
    memcpy(T, s->torque, sizeof(double) * 3 * (size_t)s->np);
}

void orc_get_solid(const orc_sim *s, int *out) { memcpy(out, s->solid, sizeof(int) * (size_t)s->n); }

void orc_get_eps(const orc_sim *s, int p, double *out) {
    memcpy(out, s->eps + (size_t)p * s->n, sizeof(double) * (size_t)s->n);
}

/* Macroscopic fields of the current pre-collision state: Eq. (4) and Eq. (8)
 * for fluid cells, Eq. (27) for PSM; MEM solid cells report rho0 and the
 * body velocity at the cell centre. */
void orc_get_macro(const orc_sim *s, double *rho_out, double *u_out) {
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = cell_index(s, x, y, z);
                double fc[NQ], rho, U[3], u[3], xc[3];
                cell_centre(x, y, z, xc);
                if (is_mem(s->p.coupling) && s->solid[i]) {
                    body_velocity(s, &s->part[s->solid[i] - 1], xc, u);
                    rho_out[i] = s->p.rho0;
                    for (int a = 0; a < 3; ++a) u_out[3 * i + a] = u[a];
                    continue;
                }
                for (int q = 0; q < NQ; ++q) fc[q] = s->f[(long)q * s->n + i];
                moments(fc, s->p.rho0, &rho, U);
                for (int a = 0; a < 3; ++a) u[a] = U[a] + s->p.fext[a] / (2.0 * s->p.rho0);
                if (is_psm(s->p.coupling)) {
                    double B = 0.0, vsum[3] = {0.0, 0.0, 0.0};
                    for (int p = 0; p < s->np; ++p) {
                        double e = s->eps[(size_t)p * s->n + i];
                        if (e <= 0.0) continue;
                        double Bs = (s->p.coupling == ORC_PSM_M1B1)
                                        ? e
                                        : e * (s->p.tau - 0.5) / ((1.0 - e) + (s->p.tau - 0.5));
                        double vs[3];
                        body_velocity(s, &s->part[p], xc, vs);
                        B += Bs;
                        for (int a = 0; a < 3; ++a) vsum[a] += Bs * vs[a];
                    }
                    for (int a = 0; a < 3; ++a) u[a] = (1.0 - B) * u[a] + vsum[a];
                }
                rho_out[i] = rho;
                for (int a = 0; a < 3; ++a) u_out[3 * i + a] = u[a];
            }
}

/* One global time step: Algorithm 2 (PSM), Algorithm 1 (MEM) or a plain
 * fluid step (no coupling). */
static int one_step(orc_sim *s) {
    int c = s->p.coupling, np = s->np;
    if (is_psm(c)) {
        /* Algorithm 2 has one LBM sweep per step; Sec. 4.1 runs two LBM
         * subcycles with the forces averaged for its settling benchmark (R30):
         * every sweep uses the particle state of the start of the step. */
        int sub = s->p.subcycles;
        for (int k = 0; k < 3 * np; ++k) { s->fsum[k] = 0.0; s->tsum[k] = 0.0; }
        compute_solid_fractions(s);
        for (int it = 0; it < sub; ++it) {
            double *F = s->force, *T = s->torque;
            for (int k = 0; k < 3 * np; ++k) { F[k] = 0.0; T[k] = 0.0; }
            collide_psm(s, F, T);
            stream(s);
            for (int k = 0; k < 3 * np; ++k) { s->fsum[k] += F[k]; s->tsum[k] += T[k]; }
        }
        for (int k = 0; k < 3 * np; ++k) {
            s->force[k] = s->fsum[k] / sub;
            s->torque[k] = s->tsum[k] / sub;
        }
        int st = rigid_body_update(s, (double)sub);
        compute_solid_fractions(s); /* keep eps in step with the current particle state */
        return st;
    }
    if (is_mem(c)) {
        if (!s->mapped) { map_particles(s, s->solid); s->mapped = 1; }
        int sub = s->p.subcycles;
        for (int k = 0; k < 3 * np; ++k) { s->fsum[k] = 0.0; s->tsum[k] = 0.0; }
        for (int it = 0; it < sub; ++it) {
            double *F = s->force, *T = s->torque;
            for (int k = 0; k < 3 * np; ++k) { F[k] = 0.0; T[k] = 0.0; }
            collide_fluid(s);
            mem_boundary(s);
            stream(s);
            mem_link_forces(s, F, T);
            for (int k = 0; k < 3 * np; ++k) { s->fsum[k] += F[k]; s->tsum[k] += T[k]; }
        }
        for (int k = 0; k < 3 * np; ++k) {
            s->force[k] = s->fsum[k] / sub;
            s->torque[k] = s->tsum[k] / sub;
        }
        if (s->p.remap_charge) /* R32 */
            for (int p = 0; p < np; ++p)
                for (int a = 0; a < 3; ++a) {
                    s->force[3 * p + a] -= s->charge[6 * p + a] / sub;
                    s->torque[3 * p + a] -= s->charge[6 * p + 3 + a] / sub;
                }
        int st = rigid_body_update(s, (double)sub);
        remap_and_refill(s, 1, s->p.remap_charge ? s->charge : NULL);
        return st;
    }
    collide_fluid(s);
    stream(s);
    return ORC_OK;
}

int orc_step(orc_sim *s, int nsteps) {
    for (int k = 0; k < nsteps; ++k) {
        int st = one_step(s);
        s->steps++;
        if (st != ORC_OK) return st;
    }
    return ORC_OK;
}
