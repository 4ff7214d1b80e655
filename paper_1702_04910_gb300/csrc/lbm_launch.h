// Host-side launch interface between the C-ABI layer and the kernels.
// Internal to the library; not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbmgpu {

struct Launch {
    Geom g;
    Coll<double> kd;   // FP64 collision constants
    Coll<float> kf;    // FP32 collision constants
    Coupl cp;
    DevParticle* parts;       // particle state used by this sweep
    DevParticle* parts_prev;  // state before the last rigid-body update (refill)
    double* partials;         // force/torque partials of this sweep
    int* status;
    int nostream;             // 1: stored buffer holds pre-collision f (no stream)
    int all_tiles;            // bulk kernel: process every tile (no coupling)
    int box[3];               // near-kernel tile box per particle
    dim3 block;
    cudaStream_t stream;
};

// Status bits raised by kernels (OR-ed into *status).
enum : int {
    ST_TOO_MANY_OBJECTS = 1,  // more than CELL_SLOTS particles touch a cell
    ST_DOMAIN = 2,            // a particle left the domain through a closed wall
    ST_REFILL_SOLID = 4,      // refill found no particle owning a cell (internal)
};

// storage: 0 = FP64, 1 = FP32 (arithmetic in the same precision)
cudaError_t launch_bulk(int storage, const void* src, void* dst, const Launch& L);
cudaError_t launch_near(int storage, const void* src, void* dst, const Launch& L);
cudaError_t launch_refill(int storage, const void* srcB, void* dst, const Launch& L,
                          const DevParticle* p_old, const DevParticle* p_new, int extrapolate);
cudaError_t launch_macro(int storage, const void* state, const Launch& L, int what, void* out);
cudaError_t launch_init_eq(int storage, void* dst, const Launch& L, double rho, double ux,
                           double uy, double uz);
cudaError_t launch_from_f64(int storage, const double* in, void* dst, long long count,
                            cudaStream_t s);
cudaError_t launch_finalize(const Launch& L, int nsub, double* force_out);
cudaError_t launch_regions(const Launch& L);
cudaError_t launch_rigid_body(const Launch& L, const double* force, double gx, double gy,
                              double gz, double dt, int wall_contact);

}  // namespace lbmgpu
