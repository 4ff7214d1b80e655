// Host-side launch interface between the C-ABI layer and the kernels.
// Internal to the library; not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>

#include "../../include/lbm_gb300.h"
#include "lbm_device.cuh"
#include "lbm_dfloat.cuh"
#include "lbm_fixed.cuh"

namespace lbmgpu {

struct Launch {
    Geom g;
    Coll<double> kd;   // FP64 collision constants
    Coll<float> kf;    // FP32 collision constants
    Coll<dfloat> kff;  // float-float collision constants (FP64 storage)
    Coll<fx64> kfx;    // fixed-point collision constants (FP64 storage)
    Coupl cp;
    DevParticle* parts;       // particle state used by this sweep
    DevParticle* parts_prev;  // state before the last rigid-body update (refill)
    double* partials;         // force/torque partials of this sweep
    int* status;
    int nostream;             // 1: stored buffer holds pre-collision f (no stream)
    int all_tiles;            // bulk kernel: process every tile (no coupling)
    int box[3];               // near-kernel grid per particle (blocks per axis)
    unsigned short* map;      // per-step geometry map (see k_map)
    int map_ext[3];           // region box extents of the map (cells)
    dim3 block;
    cudaStream_t stream;
};

// Near-kernel block shape and grid: a particle's cell region spans at most
// D + 2 NEAR_HALO + 1 cells per axis; the grid covers ceil(D) + 6 cells.
constexpr int NEAR_BX = 32, NEAR_BY = 2, NEAR_BZ = 1;
// threads per block of the refill kernels (whole warps: a warp rebuilds a cell)
constexpr int REFILL_THREADS = 128;
static_assert(NEAR_BX * NEAR_BY * NEAR_BZ % 32 == 0, "near blocks are whole warps");
static_assert(REFILL_THREADS % 32 == 0, "refill blocks are whole warps");
// blocks of the refill kernel per particle for a box of side^3 cells
__host__ __device__ inline long long refill_blocks(int side) {
    return ((long long)side * side * side + REFILL_THREADS - 1) / REFILL_THREADS;
}

// Cells per axis of the region box that holds any particle of diameter <= maxd.
inline void region_extent(const Geom& g, double maxd, int ext[3]) {
    const int span = (int)ceil(maxd) + 2 * (int)NEAR_HALO + 2;
    ext[0] = g.nx < span ? g.nx : span;
    ext[1] = g.ny < span ? g.ny : span;
    ext[2] = g.nz < span ? g.nz : span;
}

inline void near_grid(const Geom& g, double maxd, int box[3]) {
    int ext[3];
    region_extent(g, maxd, ext);
    const int b[3] = {NEAR_BX, NEAR_BY, NEAR_BZ};
    for (int a = 0; a < 3; ++a) box[a] = (ext[a] + b[a] - 1) / b[a];
}

// Map entries (unsigned short) for np particles.
inline long long map_entries(const Geom& g, double maxd, int np) {
    int ext[3];
    region_extent(g, maxd, ext);
    return (long long)(np > 0 ? np : 1) * ext[0] * ext[1] * ext[2];
}

inline long long near_blocks(const int box[3]) { return (long long)box[0] * box[1] * box[2]; }

// Doubles of force partials one sweep needs: np regions x blocks x np x 6.
inline long long near_partial_doubles(const int box[3], int np) {
    const long long n = np > 0 ? np : 1;
    return n * near_blocks(box) * n * 6;
}

// ---- batched ensemble ----------------------------------------------------------
// One independent simulation of a batch (one particle, FP64 PDFs).  Lives in
// device memory; the kernels read buf[cur] and flip cur themselves, so one
// step's launches are the same every step and can be replayed as a graph.
struct BatchCase {
    Geom g;
    double* buf[2];
    int cur;
    int kind;          // 1 PSM, 2 MEM, 0 none
    int subcycles;     // LBM sweeps per global step
    int layout;        // bulk tiling: 0 box tiles (g.tx x g.ty), 1 256-cell plane segments
    int wall_contact;
    Coupl cp;          // np = 1
    Coll<double> kd;
    Coll<fx64> kfx;
    DevParticle* part;
    DevParticle* prev;
    double* force;     // 6 doubles
    double* partials;  // subcycles x nblk x 6
    unsigned short* map;
    int map_ext[3];
    int box[3];        // near-kernel grid (blocks)
    long long nblk;
    int refill_side;
    double gravity[3];
    int remap_charge;     // MEM: charge the re-mapping momentum (lbm_batch_set_remap_charge)
    double* charge;       // 6 doubles: pending amounts of the last re-mapping
    double* charge_part;  // refill_blocks(refill_side) x 6 block partials
};

// Work list of a batched launch: cases list[0..n) with prefix sums base[] of
// their work items (tiles, blocks or cells).
struct BatchList {
    const int* list;
    const long long* base;  // n + 1 entries
    int n;
};

// Collision constants of Eq. (5) / (9)-(11) with the forcing of Eq. (7)
// (computed in FP64, rounded once to C).
// MEM MR, Eq. (15): Lambda_- = 1/|lambda_-| - 1/2 of the collision (TRT:
// Lambda / (tau - 1/2), Eq. (11); BGK: tau - 1/2).  The correction term
// f^pc = -8 Lambda_- n^-_q / ((2 Lambda_- + 1)(1 + delta)^2) needs the
// pre-collision odd non-equilibrium n^-_q(x, t); the kernels rebuild it from
// the stored post-collision values, (1 - |lambda_-|) n^-_q =
// (f~_q - f~_qbar)/2 - 3 w_q c_q . j~ (the forcing drops out), so the scale
// applied to that difference is -4 Lambda_- / (Lambda_- - 1/2).  The rebuild
// loses n^- as |lambda_-| -> 1; MR is refused within 0.01 of Lambda_- = 1/2.
inline double mr_lambda_minus(const lbm_config& cfg) {
    return cfg.collision == LBM_TRT ? cfg.magic / (cfg.tau - 0.5) : cfg.tau - 0.5;
}
inline bool mr_supported(const lbm_config& cfg) {
    return std::fabs(mr_lambda_minus(cfg) - 0.5) >= 0.01;
}
inline double mr_correction_scale(const lbm_config& cfg) {
    const double Lm = mr_lambda_minus(cfg);
    return -4.0 * Lm / (Lm - 0.5);
}

template <typename C>
inline Coll<C> make_coll(double lp, double lm, double rho0, const double fe[3]) {
    Coll<C> k{};
    k.lam_p = (C)lp;
    k.lam_m = (C)lm;
    k.rho0 = (C)rho0;
    k.inv_rho0 = (C)(1.0 / rho0);
    k.fx = (C)fe[0];
    k.fy = (C)fe[1];
    k.fz = (C)fe[2];
    k.has_force = (fe[0] != 0.0 || fe[1] != 0.0 || fe[2] != 0.0);
    k.alpha = (C)(1.0 + 0.5 * (lp + lm));
    k.beta = (C)(0.5 * (lp - lm));
    k.hs = (C)(0.5 * (1.0 + lp));
    k.hd = (C)(0.5 * (1.0 + lm));
    k.c0 = (C)(1.0 + lp);
    k.m15r0 = (C)(-1.5 / rho0);
    const double w[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    for (int c = 0; c < 3; ++c) {
        k.lpw[c] = (C)(lp * w[c]);
        k.k1w[c] = (C)(4.5 * lp * w[c] / rho0);
        k.k2w[c] = (C)(3.0 * lm * w[c]);
        k.hw[c] = (C)(3.0 * w[c] / rho0);
    }
    for (int q = 1; q < NQ; q += 2) {
        const double cf = cx(q) * fe[0] + cy(q) * fe[1] + cz(q) * fe[2];
        k.gq[(q - 1) / 2] = (C)(9.0 * wq(q) * cf / rho0);
        k.fq[(q - 1) / 2] = (C)(3.0 * wq(q) * cf);
    }
    return k;
}

// Checks of a configuration shared by every entry point that takes one
// (lbm_create, lbm_sweep_noalloc): LBM_ERR_ARG for a value outside its
// range, LBM_ERR_UNSUPPORTED for MEM MR within 0.01 of Lambda_- = 1/2.
// Host-only; touches no device state.
inline lbm_status check_config(const lbm_config& c) {
    if (c.nx < 1 || c.ny < 1 || c.nz < 1) return LBM_ERR_ARG;
    if ((long long)c.nx * c.ny * c.nz > (1LL << 40)) return LBM_ERR_ARG;
    if (!(c.tau > 0.5) || !std::isfinite(c.tau) || !(c.rho0 > 0.0) || !std::isfinite(c.rho0))
        return LBM_ERR_ARG;
    if (c.coupling < 0 || c.coupling > LBM_NONE) return LBM_ERR_ARG;
    if (c.collision != LBM_BGK && c.collision != LBM_TRT) return LBM_ERR_ARG;
    if (c.storage < LBM_STORE_F64 || c.storage > LBM_STORE_BF16S) return LBM_ERR_ARG;
    if (c.bc_z < 0 || c.bc_z > 2 || (c.bc_z == 2 && c.nz < 3)) return LBM_ERR_ARG;
    if (c.bc_z == 2 && !(std::isfinite(c.inflow[0]) && std::isfinite(c.inflow[1]) &&
                         std::isfinite(c.inflow[2]) && c.rho_out > 0.0 && std::isfinite(c.rho_out)))
        return LBM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(c.force_density[a]) || !std::isfinite(c.gravity[a])) return LBM_ERR_ARG;
    if (c.subsample < 0 || c.subsample > 40 || c.lbm_subcycles < 0) return LBM_ERR_ARG;
    if (c.collision == LBM_TRT) {
        // Eq. (11): lambda_- from Lambda = magic; it must lie in (-2, 0)
        const double lp = -1.0 / c.tau;
        const double denom = c.magic / (0.5 + 1.0 / lp) - 0.5;
        if (!(c.magic > 0.0) || !std::isfinite(c.magic) || denom == 0.0) return LBM_ERR_ARG;
        const double lm = 1.0 / denom;
        if (!(lm > -2.0 && lm < 0.0)) return LBM_ERR_ARG;
    }
    if (c.coupling == LBM_MEM_MR && !mr_supported(c)) return LBM_ERR_UNSUPPORTED;
    return LBM_OK;
}

// Open-boundary data of a configuration (bc_z = 2) into the geometry.
inline void set_open_boundaries(Geom& g, const lbm_config& cfg) {
    for (int a = 0; a < 3; ++a) {
        g.uin[a] = cfg.bc_z == 2 ? cfg.inflow[a] : 0.0;
        g.fhalf[a] = cfg.force_density[a] / (2.0 * cfg.rho0);
    }
    g.rho_out = cfg.bc_z == 2 ? cfg.rho_out : cfg.rho0;
    g.rho0 = cfg.rho0;
}

// Status bits raised by kernels (OR-ed into *status).
enum : int {
    ST_TOO_MANY_OBJECTS = 1,  // more than CELL_SLOTS particles touch a cell
    ST_DOMAIN = 2,            // a particle left the domain through a closed wall
    ST_REFILL_SOLID = 4,      // refill found no particle owning a cell (internal)
    ST_UNSTABLE = 8,          // a particle state became non-finite or too fast
    ST_BOUNDS = 16,           // an index check in a coupling kernel failed (access skipped)
    ST_FLUID = 32,            // a fluid cell's density became non-finite or <= 0
};
static_assert((int)ST_TOO_MANY_OBJECTS == (int)LBM_STATUS_TOO_MANY_OBJECTS &&
                  (int)ST_DOMAIN == (int)LBM_STATUS_DOMAIN &&
                  (int)ST_UNSTABLE == (int)LBM_STATUS_UNSTABLE &&
                  (int)ST_BOUNDS == (int)LBM_STATUS_BOUNDS && (int)ST_FLUID == (int)LBM_STATUS_FLUID,
              "status bits of the public header");

// storage: 0 = FP64, 1 = FP32 (arithmetic in the same precision), 4 = FP16
// and 5 = BF16 shifted populations f - w_q (FP32 arithmetic); launch_bulk
// also takes 2 = FP64 storage with float-float collision and 3 = FP64
// storage with 64-bit fixed-point collision
cudaError_t launch_bulk(int storage, const void* src, void* dst, const Launch& L);
cudaError_t launch_near(int storage, const void* src, void* dst, const Launch& L);
// charge_part != nullptr: also the re-mapping momentum charge partials,
// refill_blocks(L.box[0]) blocks x 6 doubles per particle (see k_refill)
cudaError_t launch_refill(int storage, const void* srcB, void* dst, const Launch& L,
                          const DevParticle* p_old, const DevParticle* p_new, int extrapolate,
                          double* charge_part = nullptr);
// charge[p * 6 + c] = fixed-order total of the refill's charge partials
cudaError_t launch_charge_total(const Launch& L, const double* charge_part, double* charge);
cudaError_t launch_macro(int storage, const void* state, const Launch& L, int what, void* out);
cudaError_t launch_init_eq(int storage, void* dst, const Launch& L, double rho, double ux,
                           double uy, double uz);
cudaError_t launch_from_f64(int storage, const double* in, void* dst, long long count,
                            long long ncell, cudaStream_t s);
cudaError_t launch_to_f64(int storage, const void* in, double* out, long long count,
                          long long ncell, cudaStream_t s);
// charge != nullptr: the pending re-mapping momentum charge, [p][6], over nsub
// is taken off the totals
cudaError_t launch_finalize(const Launch& L, int nsub, double* force_out,
                            const double* charge = nullptr);
cudaError_t launch_regions(const Launch& L);
// batched ensemble (all cases on one stream; see lbm_batch.cu)
cudaError_t launch_batch_regions(BatchCase* cases, int n, cudaStream_t s);
cudaError_t launch_batch_map(BatchCase* cases, BatchList l, long long total, cudaStream_t s);
cudaError_t launch_batch_near(BatchCase* cases, BatchList l, long long total, int sub,
                              int* status, cudaStream_t s);
// mode 0 FP64 / 3 fixed-point collision; grid <= 0: one block per tile
cudaError_t launch_batch_bulk(int mode, BatchCase* cases, BatchList l, long long total, int grid,
                              int* status, cudaStream_t s);
cudaError_t launch_batch_swap(BatchCase* cases, BatchList l, cudaStream_t s);
cudaError_t launch_batch_finalize(BatchCase* cases, int n, cudaStream_t s);
cudaError_t launch_batch_rigid(BatchCase* cases, int n, int* status, cudaStream_t s);
// p[0] = now (end = 0); p[1] += now - p[0], p[2] += 1 (end = 1); now from
// the global nanosecond timer
cudaError_t launch_stamp(unsigned long long* p, int end, cudaStream_t s);
// per case with the charge on: total of its refill-block charge partials
cudaError_t launch_batch_charge_total(BatchCase* cases, int n, cudaStream_t s);
cudaError_t launch_batch_refill(BatchCase* cases, BatchList l, long long total, int* status,
                                cudaStream_t s);
cudaError_t launch_batch_init(BatchCase* cases, int n, long long max_cells, cudaStream_t s);
int batch_bulk_blocks_per_sm(int mode);
cudaError_t launch_map(const Launch& L);
// learned force correction (lbm_learned.cu)
cudaError_t launch_features(int storage, const void* state, const Launch& L, const double* force,
                            double u_ref, float* feat);
cudaError_t launch_apply_correction(const float* y, const DevParticle* parts, int np, double u_ref,
                                    double rho0, double* force, cudaStream_t s);
// clip > 0: samples with a normalised input beyond +-clip get y = 0
cudaError_t mlp_infer(const lbm_mlp* m, const float* x, int n, float* y, float clip,
                      cudaStream_t s);
cudaError_t launch_rigid_body(const Launch& L, const double* force, double gx, double gy,
                              double gz, double dt, int wall_contact);

}  // namespace lbmgpu
