/*
 * lbm_gb300.h -- C ABI of the GB300 (sm_103a) coupled D3Q19 lattice
 * Boltzmann library.
 *
 * The library computes the coupled time step of Rettinger & Ruede,
 * "A comparative study of fluid-particle coupling methods for fully resolved
 * lattice Boltzmann simulations" (arXiv:1702.04910): a D3Q19 lattice
 * Boltzmann sweep (Sec. 2.1, Eq. (1)-(11)) fused with one of two fluid-
 * particle couplings:
 *   - PSM, partially saturated cells (Sec. 2.3, Eq. (20)-(29), Algorithm 2),
 *     variants M1B1, M2B2, M3B2;
 *   - MEM, momentum exchange (Sec. 2.2, Eq. (12)-(19), Algorithm 1),
 *     boundary schemes BB, CLI and MR (Eq. (12), (14), (15); the MR
 *     coefficients, only cited by the paper, are derived for the TRT link
 *     recurrence, see LBM_MEM_MR);
 * followed by the per-particle force/torque reduction and an explicit
 * rigid-body update of spherical particles.
 *
 * Conventions shared by every entry point:
 *   - Lattice units: dx = dt = 1.  Cell (x,y,z) has its centre at
 *     (x+1/2, y+1/2, z+1/2); the domain is [0,nx) x [0,ny) x [0,nz),
 *     periodic in x and y, periodic or closed (resting no-slip walls at
 *     z = 0 and z = nz) in z.
 *   - PDF fields are structure-of-arrays, index q*N + x + nx*(y + ny*z) with
 *     N = nx*ny*nz and q in the order: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z;
 *     7..18 = (+1,+1,0),(-1,-1,0),(+1,-1,0),(-1,+1,0),(+1,0,+1),(-1,0,-1),
 *     (+1,0,-1),(-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1).
 *   - The handle owns all device memory it allocates.  Every buffer passed in
 *     is owned by the caller and only read or written during the call (or,
 *     for device pointers, in stream order on the handle's stream).
 *   - Work is enqueued on the CUDA stream given to lbm_create (the legacy
 *     default stream if NULL).  Calls that return data to host memory
 *     synchronise that stream.
 *   - No C++ exception crosses this interface.  Every call returns an
 *     lbm_status; on failure lbm_last_error() describes the cause.  Device
 *     kernels never trap: they raise a status word that the next
 *     synchronising call (lbm_get_forces, lbm_get_particles, lbm_get_fields,
 *     lbm_synchronize) reports.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,         /* invalid argument; nothing was changed            */
    LBM_ERR_CUDA = -2,        /* a CUDA runtime call failed                       */
    LBM_ERR_OOM = -3,         /* device or pinned host allocation failed          */
    LBM_ERR_UNSTABLE = -4,    /* a particle state became non-finite or moved a    */
                              /* cell or more per step (update not applied), or a */
                              /* fluid cell's density became non-finite or <= 0   */
    LBM_ERR_DOMAIN = -5,      /* a particle left the domain through a closed wall */
    LBM_ERR_TIMEOUT = -6,     /* reserved: a bounded device wait gave up          */
    LBM_ERR_UNSUPPORTED = -7  /* configuration not implemented (e.g. MR near |lambda_-| = 1) */
} lbm_status;

/* Coupling of Sec. 2.2 / 2.3.  LBM_NONE runs the plain fluid sweep. */
typedef enum {
    LBM_PSM_M1B1 = 0, /* Eq. (21) with Eq. (23)                      */
    LBM_PSM_M2B2 = 1, /* Eq. (22) with Eq. (24)                      */
    LBM_PSM_M3B2 = 2, /* Eq. (22) with Eq. (25)                      */
    LBM_MEM_BB = 3,   /* Eq. (12)                                    */
    LBM_MEM_CLI = 4,  /* Eq. (14)                                    */
    LBM_MEM_MR = 5,   /* Eq. (15) multi-reflection.  The paper cites its coefficients;
                       * here they are derived from the second-order no-slip
                       * requirement on the steady TRT link recurrence:
                       * kappa_1 = 1, kappa_0 = (1-2d-2d^2)/(1+d)^2,
                       * kappa_-1 = d^2/(1+d)^2, kappabar_-1 = -kappa_0,
                       * kappabar_-2 = -kappa_-1, alpha = 4/(1+d)^2,
                       * f^pc = -8 Lambda_- n^-_q(x,t) / ((2 Lambda_- + 1)(1+d)^2)
                       * with d = delta_q and n^-_q the odd pre-collision
                       * non-equilibrium at x, rebuilt from the stored
                       * post-collision values.  Needs x - c_q and x - 2 c_q
                       * fluid (else CLI, else BB).  Refused (LBM_ERR_UNSUPPORTED)
                       * when |Lambda_- - 1/2| < 0.01, Lambda_- = Lambda/(tau-1/2)
                       * (TRT) or tau - 1/2 (BGK), where the rebuild loses n^-. */
    LBM_NONE = 6
} lbm_coupling;

/* Fluid collision operator: BGK Eq. (5) or TRT Eq. (9)-(11). */
typedef enum { LBM_BGK = 0, LBM_TRT = 1 } lbm_collision;

/* PDF storage and collision arithmetic.  Forces, solid fractions and the
 * rigid-body update are FP64 in every mode.
 *   LBM_STORE_F64     FP64 PDFs, FP64 arithmetic.
 *   LBM_STORE_F32     FP32 PDFs, FP32 collision arithmetic.
 *   LBM_STORE_F64_FF  FP64 PDFs; the collision of cells away from particles
 *                     runs in float-float arithmetic (a value is the sum of
 *                     two floats, ~48 significant bits, converted from and to
 *                     FP64 with integer operations); cells near particles
 *                     use FP64.  Same state layout as LBM_STORE_F64.
 *   LBM_STORE_F64_FX  FP64 PDFs; the collision of cells away from particles
 *                     runs in 64-bit fixed point (value = integer * 2^-58:
 *                     exact sums, products to 2^-58), converted from and to
 *                     FP64 with integer operations; cells near particles use
 *                     FP64.  Same state layout as LBM_STORE_F64.
 *   LBM_STORE_F16S    PDFs stored as FP16 shifted populations f_q - w_q, FP32
 *                     collision arithmetic (76 B per cell update).
 *   LBM_STORE_BF16S   the same with BF16 storage. */
typedef enum {
    LBM_STORE_F64 = 0,
    LBM_STORE_F32 = 1,
    LBM_STORE_F64_FF = 2,
    LBM_STORE_F64_FX = 3,
    LBM_STORE_F16S = 4,
    LBM_STORE_BF16S = 5
} lbm_storage;

typedef struct {
    int nx, ny, nz;            /* cells per axis, each >= 1                        */
    int bc_z;                  /* 0: periodic in z; 1: resting no-slip walls;     */
                               /* 2: the open boundaries of Sec. 4.1: velocity    */
                               /*    bounce-back (Eq. (12)) with `inflow` at      */
                               /*    z = 0, outflow f_qbar = -f~_q + 2 f_eq,+_q(  */
                               /*    rho_out, u) at z = nz; a particle must stay  */
                               /*    R + 3 cells away from both (LBM_ERR_DOMAIN)  */
    int collision;             /* lbm_collision                                   */
    int coupling;              /* lbm_coupling                                    */
    double tau;                /* relaxation time, > 1/2 (nu = (tau - 1/2)/3)     */
    double magic;              /* TRT Lambda of Eq. (11), e.g. 3/16               */
    double force_density[3];   /* f_ext of Eq. (7), acts on the fluid             */
    double gravity[3];         /* acceleration acting on the particles            */
    double rho0;               /* reference density rho_0 (> 0)                   */
    int subsample;             /* PSM: n of the n^3 supersampling (0 -> 4)        */
    int lbm_subcycles;         /* LBM sweeps per global step, forces averaged over */
                               /* them (0 -> 2 MEM, 1 PSM; PSM 2: Sec. 4.1)      */
    int wall_contact;          /* 1: keep spheres one cell off closed z walls     */
    int storage;               /* lbm_storage                                     */
    double inflow[3];          /* bc_z = 2: inflow velocity at z = 0              */
    double rho_out;            /* bc_z = 2: outflow density at z = nz             */
} lbm_config;

/* Rigid spherical particle (Eq. (13) velocity field). */
typedef struct {
    double x[3];       /* centre X_p                                 */
    double u[3];       /* translational velocity U_p                 */
    double omega[3];   /* angular velocity Omega_p                   */
    double diameter;   /* D                                          */
    double density;    /* rho_p                                      */
    int fixed;         /* 1: position and velocity are held constant */
} lbm_particle;

typedef struct lbm_handle lbm_handle;

/* Field selectors of lbm_get_fields / lbm_set_fields. */
enum {
    LBM_FIELD_PDF = 0,     /* stored post-collision PDFs (state), 19*N of the storage type
                              (FP16/BF16 modes: the shifted values f_q - w_q) */
    LBM_FIELD_PDF_PRE = 1, /* set only: pre-collision PDFs f at t = 0, 19*N doubles        */
    LBM_FIELD_RHO = 2,     /* get only: fluid density rho_f, N doubles                     */
    LBM_FIELD_U = 3,       /* get only: velocity u, Eq. (8) / (27), 3*N doubles [cell][3]   */
    LBM_FIELD_EPS = 4,     /* get only: PSM solid fraction sum_s eps_s, N doubles          */
    LBM_FIELD_FLAG = 5,    /* get only: MEM owner (0 fluid, s+1 inside particle s), N int32 */
    LBM_FIELD_PDF_F64 = 6, /* get only: the stored PDFs as FP64 values of f (shift undone) */
    LBM_FIELD_REMAP_CHARGE = 7 /* MEM: the pending re-mapping momentum charge (see
                              lbm_set_remap_charge), 6*n_particles doubles [p][Px Py Pz
                              Lx Ly Lz]; part of a checkpoint when the charge is on */
};

/* Create a simulation.  Validates *cfg (LBM_ERR_ARG on a bad value,
 * LBM_ERR_UNSUPPORTED for LBM_MEM_MR with |Lambda_- - 1/2| < 0.01),
 * allocates two PDF buffers of
 * 19*N elements on the current CUDA device and initialises the fluid at rest
 * (f = f_eq(rho0, 0), Eq. (3)).  stream: a cudaStream_t or NULL.
 * On success *out receives the handle; release it with lbm_destroy. */
lbm_status lbm_create(const lbm_config *cfg, void *stream, lbm_handle **out);

/* Replace the particle state with n host records (n <= 32; D >= 1 and D + 4
 * cells below each periodic extent).  Before the first step this defines the
 * initial mapping (MEM, Sec. 2.2) and the solid fractions (PSM, Sec. 2.3).
 * Between steps with MEM coupling, cells uncovered by the replacement are
 * refilled with f_eq(rho0, v) (the particle count must not change then). */
lbm_status lbm_set_particles(lbm_handle *h, int n, const lbm_particle *host_in);

/* Copy the current particle state into host_out (n records). Synchronises. */
lbm_status lbm_get_particles(lbm_handle *h, lbm_particle *host_out);

/* Set the pre-collision state at t = 0 to f_eq(rho, u) in every cell, Eq. (3). */
lbm_status lbm_init_equilibrium(lbm_handle *h, double rho, const double u[3]);

/* Advance nsteps global time steps (Algorithm 1 for MEM, Algorithm 2 for
 * PSM).  Each step runs lbm_subcycles LBM sweeps with the particle state of
 * its start (MEM default 2; PSM default 1, or 2 as in the settling benchmark
 * of Sec. 4.1), averages their forces and advances the particles by
 * dt = lbm_subcycles.  Asynchronous: returns after enqueueing. */
lbm_status lbm_step(lbm_handle *h, int nsteps);

/* Hydrodynamic force and torque of the last global step, Eq. (17)-(18)
 * (MEM) or Eq. (28)-(29) (PSM), averaged over the step's subcycles (MEM with
 * lbm_set_remap_charge on: minus the pending re-mapping charge over dt).  F and T are
 * host arrays of 3*n doubles [particle][3].  Synchronises and reports any
 * device status raised since the last synchronising call. */
lbm_status lbm_get_forces(lbm_handle *h, double *F, double *T);

/* Copy a field (see LBM_FIELD_*) into dst, a host or device buffer of
 * exactly `bytes` bytes (LBM_ERR_ARG otherwise).  RHO/U/EPS/FLAG describe
 * the pre-collision state at the start of the next step.  Synchronises. */
lbm_status lbm_get_fields(lbm_handle *h, int what, void *dst, size_t bytes, int dst_is_device);

/* Overwrite a field from src (host or device, exactly `bytes` bytes).
 * LBM_FIELD_PDF restores a state saved with lbm_get_fields (checkpoint);
 * LBM_FIELD_PDF_PRE sets the pre-collision PDFs at t = 0. */
lbm_status lbm_set_fields(lbm_handle *h, int what, const void *src, size_t bytes, int src_is_device);

/* MEM re-mapping momentum charge, off by default (Algorithm 1 of the paper
 * has no such step; the option is this library's).  The re-mapping at the
 * end of a MEM step (Sec. 2.2) removes from the fluid the momentum
 * sum_q c_q f_q of every cell a particle covers and creates that of every
 * cell it uncovers (the populations rebuilt by Eq. (19)).  With enable = 1
 * the difference dP (created minus removed) and its moment dL about the
 * particle's new centre are kept per particle, and the next step's averaged
 * force and torque become F - dP/dt and T - dL/dt (dt = lbm_subcycles)
 * before the rigid-body update.  A sphere that crosses the lattice then
 * feels the drag of the same sphere held in a uniform stream; without the
 * charge it feels less (the finer the lattice, the smaller the gap).
 * Switching, and lbm_set_particles, clear the pending amounts.  The charge
 * covers cells within the refill box, which holds the new sphere while its
 * centre moves less than 1.5 cells per axis in a step (a faster step raises
 * LBM_ERR_UNSTABLE).  LBM_ERR_UNSUPPORTED for a PSM or uncoupled handle
 * with enable = 1; LBM_ERR_ARG for enable other than 0 or 1. */
lbm_status lbm_set_remap_charge(lbm_handle *h, int enable);

/* Wait for all enqueued work and report device status. */
lbm_status lbm_synchronize(lbm_handle *h);

/* Per-kernel device timing with CUDA events on the handle's stream.
 * lbm_profile_enable(h, 1) starts recording (and clears the totals);
 * lbm_profile_read returns, for each kernel class k < n_classes
 * (0 bulk sweep, 1 near-particle sweep, 2 force reduction, 3 rigid-body
 * update, 4 MEM refill, 5 other: per-step geometry map and set-up
 * collisions), the summed milliseconds and launches.
 * Reading synchronises the stream. */
lbm_status lbm_profile_enable(lbm_handle *h, int enable);
lbm_status lbm_profile_read(lbm_handle *h, int n_classes, double *ms, long long *launches);

/* Bytes of device memory held by the handle. */
size_t lbm_device_bytes(const lbm_handle *h);

/* Release every resource of the handle (NULL is ignored). */
void lbm_destroy(lbm_handle *h);

/* Human-readable description of the last failure on h ("" if none; a
 * static string for h == NULL). */
const char *lbm_last_error(const lbm_handle *h);

/* Measurement utility; the paper has no counterpart.  The FP64 sweep is
 * bound by the rate at which the GPU issues FP64 instructions, so its
 * roofline needs that rate measured on the device.  Runs independent chains
 * of FP64 fused multiply-adds on every SM of the current device (stream: a
 * cudaStream_t or NULL), times them with CUDA events (best of three launches
 * after a warm-up, a few milliseconds in all) and stores the DFMA
 * lane-operations per second in *dfma_per_second (one DFMA = 2 flops).
 * Synchronises the stream.  LBM_ERR_ARG for a NULL output, LBM_ERR_CUDA when
 * a CUDA call fails (the output is then 0). */
lbm_status lbm_measure_fp64_rate(void *stream, double *dfma_per_second);

/* ABI version of this header: 1. */
int lbm_abi_version(void);

/* Bits the kernels OR into a device status word (lbm_sweep_noalloc's
 * status_dev; the handle and the batch map them to return codes). */
enum {
    LBM_STATUS_TOO_MANY_OBJECTS = 1, /* more than two particles touch one cell          */
    LBM_STATUS_DOMAIN = 2,           /* a particle left through a closed wall           */
    LBM_STATUS_UNSTABLE = 8,         /* a particle state became non-finite or too fast  */
    LBM_STATUS_BOUNDS = 16,          /* an index check in a coupling kernel failed      */
    LBM_STATUS_FLUID = 32            /* a fluid cell's density became non-finite or <= 0 */
};

/* Capacity, in doubles, of the fixed force-partial scratch that
 * lbm_sweep_noalloc uses: 524288 doubles = 4 MiB per GPU. */
#define LBM_NOALLOC_MAX_PARTIAL_DOUBLES 524288

/* One coupled LBM sweep that allocates no memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc / cudaFree while they step -- a host program that owns every
 * device byte through its own arena or pool, or a time-stepping loop that
 * cannot take the implicit device-wide synchronisation cudaFree (and at
 * times cudaMalloc) performs while other streams are busy.
 *
 * It performs what one sweep of lbm_step does on a handle: pull stream,
 * collision and coupling (PSM or MEM, cfg->coupling) of FP64 PDFs, then the
 * fixed-order force/torque total of that sweep -- but no subcycle average,
 * rigid-body update or MEM refilling, and no handle.
 *   cfg              configuration as for lbm_create; storage must be
 *                    LBM_STORE_F64 (LBM_ERR_UNSUPPORTED otherwise); LBM_MEM_MR
 *                    is refused as in lbm_create (|Lambda_- - 1/2| < 0.01).
 *   src_pdf_dev      device, 19*N doubles: post-collision PDFs (the layout
 *                    of lbm_get_fields(LBM_FIELD_PDF)); read only.
 *   dst_pdf_dev      device, 19*N doubles, distinct from src: receives the
 *                    new post-collision PDFs (MEM solid cells are left as
 *                    they were).
 *   n, particles_host   0..32 particle records on the host (copied).
 *   force_torque_dev device, 6*n doubles [particle][Fx,Fy,Fz,Tx,Ty,Tz].
 *   status_dev       device int or NULL; kernels OR LBM_STATUS_* bits into
 *                    it (the caller zeroes it and reads it after the work
 *                    has finished).  NULL sends the bits to an internal word
 *                    that the caller cannot read, so device-side errors of
 *                    the call (an index check, more than two objects in a
 *                    cell, a fluid cell whose density became non-finite or
 *                    <= 0) are then discarded.
 *   stream           cudaStream_t or NULL; work is enqueued there and the
 *                    call returns after enqueueing.  It waits for nothing:
 *                    the particle records reach the device as a kernel
 *                    argument.
 *   err, err_len     optional buffer for a message on failure.
 * Scratch: the force partials of the near-particle blocks live in a fixed
 * device array of LBM_NOALLOC_MAX_PARTIAL_DOUBLES doubles, next to a
 * geometry map of 1,048,576 16-bit entries (2 MiB), 32 particle records and
 * a status word; every GPU using the library holds them until exit.  A call
 * needs max(n,1)^2 * B * 6 doubles of partials, where B = ceil(E_x/32) *
 * ceil(E_y/2) * E_z and E_a = min(ceil(D_max) + 6, extent of axis a), and
 * max(n,1) * E_x * E_y * E_z map entries; a request beyond either capacity
 * (e.g. more than 13 spheres of D = 24) returns LBM_ERR_ARG with a message
 * saying so, before any device work is enqueued.
 * All calls share that scratch and it keeps the last call's contents, so
 * calls that may overlap on the GPU (different streams, or threads without
 * ordering) race and must be serialised by the caller.
 * The first call on each device looks up the scratch's device address with
 * cudaGetSymbolAddress (the device must be current); make that first call
 * before any stream capture.  Nothing is allocated, by this call or by any
 * library routine it calls. */
lbm_status lbm_sweep_noalloc(const lbm_config *cfg, const double *src_pdf_dev,
                             double *dst_pdf_dev, int n, const lbm_particle *particles_host,
                             double *force_torque_dev, int *status_dev, void *stream,
                             char *err, size_t err_len);

/* ---- batched ensemble -------------------------------------------------------
 * Many independent single-sphere cases (each its own lattice, configuration
 * and particle) advanced together on one GPU.  This is how ensembles of
 * settling cases (uneven domain sizes and Galileo numbers, Sec. 4 of the
 * paper studies one case at a time) are produced at full-GPU occupancy:
 *   - every kernel of a global step is one launch over all cases (work items
 *     of the cases concatenated; each block finds its case by binary search
 *     over the prefix sums of the per-case item counts);
 *   - the bulk sweep is a persistent kernel whose blocks stride over the
 *     tiles of all cases; the near-particle sweep runs beside it;
 *   - the launches of one global step are captured once into a CUDA graph
 *     and replayed by lbm_batch_step;
 *   - lbm_batch_autotune picks each case's tile layout and the bulk grid by
 *     timing them (results do not depend on the choice).
 * Each case follows the step contract of lbm_step (MEM: lbm_subcycles
 * sweeps, averaged forces, rigid-body update with dt = subcycles, refilling;
 * PSM: lbm_subcycles sweeps, default one).  The stored state of every case starts as the
 * fluid at rest, f~ = f_eq(rho0, 0) (Eq. (3)), taken as the post-collision
 * field of step 0. */
typedef struct lbm_batch lbm_batch;

/* Bulk-sweep tile layouts of lbm_batch_set_tuning. */
enum {
    LBM_BATCH_BOX32 = 0,  /* 32 x 8 cell tiles of one z plane                  */
    LBM_BATCH_BOX64 = 1,  /* 64 x 4                                            */
    LBM_BATCH_BOX128 = 2, /* 128 x 2                                           */
    LBM_BATCH_PLANE = 3   /* 256 consecutive cells of an xy plane (x fastest)  */
};

/* Creates a batch of n_cases (1..4096) cases.
 *   cfgs[c]       configuration of case c (as for lbm_create); coupling must
 *                 be a PSM or MEM variant (LBM_MEM_MR as for lbm_create);
 *                 bc_z 0 or 1; storage must be LBM_STORE_F64 or
 *                 LBM_STORE_F64_FX and the same for every case.
 *   particles[c]  the one sphere of case c (copied).
 *   stream        cudaStream_t or NULL: stream of every batch call.
 * All device memory of the batch is one allocation (PDF buffers, particle
 * records, force partials and geometry maps, 256-byte aligned slices).
 * Returns LBM_ERR_ARG for an invalid case, LBM_ERR_UNSUPPORTED for a valid
 * but unsupported one (nothing is allocated; lbm_batch_last_error(NULL) says
 * which case and why), LBM_ERR_OOM when the allocation fails. */
lbm_status lbm_batch_create(int n_cases, const lbm_config *cfgs, const lbm_particle *particles,
                            void *stream, lbm_batch **out);

/* Enqueues nsteps global steps of every case (graph replays; asynchronous). */
lbm_status lbm_batch_step(lbm_batch *b, int nsteps);

/* Autotuner.  (1) For every case, times the bulk sweep of that case alone in
 * each tile layout (LBM_BATCH_*) and keeps the fastest, so every case gets
 * its own block shape; (2) times the bulk sweep of all cases with one block
 * per tile and with persistent grids of 1x, 2x and 4x the GPU's resident
 * blocks, keeps the fastest, and rebuilds the step graph.  `reps` (1..100)
 * launches per measurement.  The timed launches write only the buffer the
 * next sweep overwrites, so the simulation state is unchanged (results do
 * not depend on the tuning).  Outputs, each may be NULL: layouts[n_cases],
 * the grid (0 = one block per tile) and the mean bulk-sweep time in ms. */
lbm_status lbm_batch_autotune(lbm_batch *b, int reps, int *layouts, int *grid, double *ms);

/* Sets the bulk layout of every case (layouts[n_cases], LBM_BATCH_*; NULL:
 * all LBM_BATCH_PLANE) and the grid (0 = one block per tile, else the number
 * of persistent blocks), then rebuilds the step graph. */
lbm_status lbm_batch_set_tuning(lbm_batch *b, const int *layouts, int grid);

/* Particle state of every case (n_cases records; synchronises). */
lbm_status lbm_batch_get_particles(lbm_batch *b, lbm_particle *host_out);

/* Hydrodynamic force and torque of the last step of every case, as for
 * lbm_get_forces: F and T each n_cases x 3 doubles (synchronises). */
lbm_status lbm_batch_get_forces(lbm_batch *b, double *F, double *T);

/* Stored post-collision PDFs of case c (19 * N_c doubles, layout of
 * LBM_FIELD_PDF) into host memory; bytes must equal 19 * N_c * 8. */
lbm_status lbm_batch_get_pdf(lbm_batch *b, int c, double *host_out, size_t bytes);

/* Lattice cell updates per global step, summed over the cases (MEM cases
 * count each sweep). */
long long lbm_batch_cell_updates(const lbm_batch *b);

/* The re-mapping momentum charge of lbm_set_remap_charge (off by default),
 * switched for every MEM case of the batch (PSM cases have no re-mapping and
 * are unaffected).  Clears the pending amounts and rebuilds the step graph
 * (one more kernel per step when on); synchronises. */
lbm_status lbm_batch_set_remap_charge(lbm_batch *b, int enable);

/* Device timing of the batch's bulk sweeps (a measurement aid; the paper has
 * no counterpart).  enable = 1 rebuilds the step graph with a one-thread
 * stamp kernel before and after every bulk-sweep launch (two more kernels
 * per LBM sweep, counted by lbm_batch_graph_kernels); they read the GPU's
 * nanosecond global timer and add each bulk sweep's span to a device
 * counter.  Enabling, or disabling, clears the counter.
 * lbm_batch_profile_read returns the summed milliseconds and the number of
 * bulk sweeps timed since then; it synchronises the stream. */
lbm_status lbm_batch_profile_enable(lbm_batch *b, int enable);
lbm_status lbm_batch_profile_read(lbm_batch *b, double *bulk_ms, long long *launches);

/* Device bytes held by the batch. */
size_t lbm_batch_device_bytes(const lbm_batch *b);

/* Number of kernel launches in one global step's graph. */
int lbm_batch_graph_kernels(const lbm_batch *b);

/* Waits for the batch's stream; reports a raised device status. */
lbm_status lbm_batch_synchronize(lbm_batch *b);

void lbm_batch_destroy(lbm_batch *b);

/* Message of the last failure on b; with b == NULL, why the calling thread's
 * last lbm_batch_create failed (empty after a success). */
const char *lbm_batch_last_error(const lbm_batch *b);

/* ---- learned force correction ----------------------------------------------
 * Not in the paper (an extension of its resolution study, Sec. 4): a small
 * MLP predicts, from a particle's near-surface stencil at coarse resolution,
 * the correction that brings the coarse run's hydrodynamic force and torque to
 * those of a finely resolved run of the same method.
 *
 * Features (LBM_MLP_IN floats per particle):
 *   [0,125)    solid indicator at a 5x5x5 grid of points X_p + (i-2, j-2,
 *              k-2) h, h = (R + 2)/2, trilinear from cell centres (PSM:
 *              min(sum_s eps_s, 1); MEM: 1 solid, 0 fluid);
 *   [125,500)  (u - U_p)/u_ref at the same points (x, y, z blocks), u = j~/rho0
 *              of the stored post-collision PDFs, body velocity in MEM solid
 *              cells, 0 beyond a closed wall;
 *   [500,512)  U_p/u_ref, Omega_p R/u_ref, F/(rho0 u_ref^2 D^2),
 *              T/(rho0 u_ref^2 D^3), with F, T this step's hydrodynamic force.
 * Outputs (LBM_MLP_OUT): (dF, dT) in the units of the last two blocks.
 * Network: x^ = (x - mu)/sigma; h1 = tanh(W1 x^ + b1); h2 = tanh(W2 h1 + b2);
 * y^ = W3 h2 + b3; y = y^ * s_out.  FP32 parameters, [in][out] layout:
 * W1 (512x64), b1, W2 (64x64), b2, W3 (64x6), b3 (LBM_MLP_PARAMS floats).
 * Normalisation block (LBM_MLP_NORM floats): mu[512], 1/sigma[512], s_out[6].
 * Loss: L = 1/(2n) sum_s sum_k w_k (y^_sk - t_sk / s_out_k)^2 with
 * w_k = (s_out_k / max_j s_out_j)^2: each output has its own scale, and its
 * error counts in the units of the largest target. */
#define LBM_MLP_IN 512
#define LBM_MLP_HIDDEN 64
#define LBM_MLP_OUT 6
#define LBM_MLP_PARAMS 37382
#define LBM_MLP_NORM 1030

typedef struct lbm_mlp lbm_mlp;

/* Creates a model (parameters zero, identity normalisation) whose kernels run
 * on `stream` (NULL: legacy default stream). */
lbm_status lbm_mlp_create(void *stream, lbm_mlp **out);
void lbm_mlp_destroy(lbm_mlp *m);
const char *lbm_mlp_last_error(const lbm_mlp *m);

/* Parameters / normalisation from or to host memory (count must equal
 * LBM_MLP_PARAMS / LBM_MLP_NORM).  Setting parameters resets Adam's moments. */
lbm_status lbm_mlp_set_params(lbm_mlp *m, const float *host, size_t count);
lbm_status lbm_mlp_get_params(lbm_mlp *m, float *host, size_t count);
lbm_status lbm_mlp_set_normalization(lbm_mlp *m, const float *host, size_t count);
lbm_status lbm_mlp_get_normalization(lbm_mlp *m, float *host, size_t count);

/* Fits the normalisation to n samples on the device: mu and 1/sigma per input
 * (sigma < 1e-6 -> 1), s_out = RMS of each target (floored at 1e-12).
 * x_dev: n x LBM_MLP_IN floats; t_dev: n x LBM_MLP_OUT floats. */
lbm_status lbm_mlp_fit_normalization(lbm_mlp *m, const float *x_dev, const float *t_dev, int n);

/* y_dev (n x LBM_MLP_OUT) = MLP(x_dev) on the device (asynchronous). */
lbm_status lbm_mlp_forward(lbm_mlp *m, const float *x_dev, int n, float *y_dev);

/* Loss and parameter gradient dL/dP over n samples (FP32, samples summed in
 * order: deterministic).  grad_host (LBM_MLP_PARAMS floats) and loss may be
 * NULL; synchronises when either is given. */
lbm_status lbm_mlp_gradient(lbm_mlp *m, const float *x_dev, const float *t_dev, int n,
                            float *grad_host, size_t count, double *loss);

/* `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, rate lr)
 * on n samples; *loss (may be NULL) receives the loss at the parameters
 * before the last update. */
lbm_status lbm_mlp_train(lbm_mlp *m, const float *x_dev, const float *t_dev, int n, int steps,
                         float lr, double *loss);

/* Attaches a force model to a handle.  mode 0: off; 1: every step computes
 * the features of each particle after the sweeps, evaluates m and adds the
 * correction to the hydrodynamic force and torque before the rigid-body
 * update (lbm_get_forces then returns the corrected values; a particle with
 * a normalised feature beyond +-10, i.e. outside the training data, keeps its
 * plain force); 2: features
 * only (no correction; m may be NULL).  u_ref > 0 is the velocity scale of
 * the features.  The model must live on the handle's device and stay alive
 * while attached. */
lbm_status lbm_set_force_model(lbm_handle *h, lbm_mlp *m, double u_ref, int mode);

/* Features of the last step (n_particles x LBM_MLP_IN floats, host;
 * synchronises).  count must equal n_particles * LBM_MLP_IN. */
lbm_status lbm_get_features(lbm_handle *h, float *host, size_t count);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
