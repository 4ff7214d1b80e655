// lbm_sweep_noalloc: one coupled LBM sweep on caller-owned device buffers
// that allocates no memory (declaration and contract in include/lbm_gb300.h).
//
// Who needs it: programs that must not call cudaMalloc / cudaFree while they
// step, e.g. a host code that owns every device byte through its own arena or
// pool, or a stepping loop that cannot afford the implicit device-wide
// synchronisation that cudaFree (and sometimes cudaMalloc) performs while
// other streams are busy.  The handle-based API allocates its buffers in
// lbm_create / lbm_set_particles; this entry point instead takes the PDF
// buffers and the force output from the caller and keeps its only scratch --
// the per-block force/torque partials, the particle records and a status
// word -- in fixed file-scope device arrays below.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/lbm_gb300.h"
#include "lbm_launch.h"

using namespace lbmgpu;

namespace {

// Scratch shared by every call on a device (held by each GPU that loads the
// library until the process exits): near-kernel force partials
// (np regions x blocks x np x 6 doubles, see near_partial_doubles), the
// per-call geometry map (np x region box entries), the particle records and
// a status word.
constexpr size_t NOALLOC_PARTIAL_DOUBLES = LBM_NOALLOC_MAX_PARTIAL_DOUBLES;
static __device__ __align__(256) double g_partials[NOALLOC_PARTIAL_DOUBLES];
static __device__ __align__(256) DevParticle g_particles[MAX_PARTICLES];
static __device__ __align__(256) int g_status[64];
constexpr size_t NOALLOC_MAP_ENTRIES = 1 << 20;  // geometry map, 2 MiB
static __device__ __align__(256) unsigned short g_map[NOALLOC_MAP_ENTRIES];

// Particle records passed by value to the kernel that stores them in
// g_particles (32 x 160 B: within the 32 KiB kernel-argument limit).
struct ParticleUpload {
    DevParticle rec[MAX_PARTICLES];
};
static_assert(sizeof(ParticleUpload) <= 32000, "kernel argument too large");

__global__ void k_upload_particles(ParticleUpload up, int n) {
    const int i = threadIdx.x;
    if (i < n && i < MAX_PARTICLES) g_particles[i] = up.rec[i];
}

constexpr int MAX_DEVICES = 64;
struct Addresses {
    bool ready;
    double* partials;
    DevParticle* particles;
    int* status;
    unsigned short* map;
};
Addresses g_addr[MAX_DEVICES];
std::mutex g_addr_mutex;

void set_err(char* err, size_t len, const char* msg) {
    if (err && len > 0) std::snprintf(err, len, "%s", msg);
}

// Device addresses of the scratch arrays on the current device, looked up
// once per device (host code cannot use the arrays' names as pointers).
cudaError_t scratch_addresses(int dev, Addresses& out) {
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    Addresses& a = g_addr[dev];
    if (!a.ready) {
        cudaError_t e = cudaGetSymbolAddress((void**)&a.partials, g_partials);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&a.particles, g_particles);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&a.status, g_status);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&a.map, g_map);
        if (e != cudaSuccess) return e;
        a.ready = true;
    }
    out = a;
    return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_sweep_noalloc(const lbm_config* cfg, const double* src_pdf_dev,
                                        double* dst_pdf_dev, int n,
                                        const lbm_particle* particles_host,
                                        double* force_torque_dev, int* status_dev, void* stream,
                                        char* err, size_t err_len) {
    if (!cfg || !src_pdf_dev || !dst_pdf_dev || src_pdf_dev == dst_pdf_dev) {
        set_err(err, err_len, "null or aliased PDF buffers");
        return LBM_ERR_ARG;
    }
    {
        // the same checks as lbm_create
        const lbm_status st = check_config(*cfg);
        if (st != LBM_OK) {
            set_err(err, err_len,
                    st == LBM_ERR_UNSUPPORTED ? "MEM MR needs |Lambda_- - 1/2| >= 0.01"
                                              : "invalid configuration");
            return st;
        }
    }
    if (cfg->storage != LBM_STORE_F64) {
        set_err(err, err_len, "lbm_sweep_noalloc takes FP64 PDF buffers only");
        return LBM_ERR_UNSUPPORTED;
    }
    const bool coupled = cfg->coupling != LBM_NONE;
    if (n < 0 || n > MAX_PARTICLES || (coupled && n > 0 && (!particles_host || !force_torque_dev))) {
        set_err(err, err_len, "particle count must be 0..32 with host records and a force output");
        return LBM_ERR_ARG;
    }
    if (!coupled) n = 0;

    Launch L{};
    Geom& g = L.g;
    g.nx = cfg->nx;
    g.ny = cfg->ny;
    g.nz = cfg->nz;
    g.bc_z = cfg->bc_z;
    g.n = (long long)cfg->nx * cfg->ny * cfg->nz;
    set_open_boundaries(g, *cfg);
    g.tx = cfg->nx >= 128 ? 128 : (cfg->nx >= 64 ? 64 : 32);
    g.ty = 256 / g.tx;
    g.ntx = (cfg->nx + g.tx - 1) / g.tx;
    g.nty = (cfg->ny + g.ty - 1) / g.ty;
    g.tz = 1;
    g.ntz = cfg->nz;
    double maxd = 0.0;
    ParticleUpload up{};
    for (int i = 0; i < n; ++i) {
        const lbm_particle& p = particles_host[i];
        const double need = p.diameter + 2.0 * NEAR_HALO + 2.0;
        const double margin = g.bc_z == 2 ? OPEN_MARGIN : 0.0;
        bool finite = std::isfinite(p.diameter) && std::isfinite(p.density);
        for (int a = 0; a < 3; ++a)
            finite = finite && std::isfinite(p.x[a]) && std::isfinite(p.u[a]) &&
                     std::isfinite(p.omega[a]);
        if (!finite || !(p.diameter >= 1.0) || !(p.density > 0.0) || need > g.nx || need > g.ny ||
            (!g.bc_z && need > g.nz) ||
            (g.bc_z && (p.x[2] - 0.5 * p.diameter - margin < 0.0 ||
                        p.x[2] + 0.5 * p.diameter + margin > g.nz))) {
            set_err(err, err_len, "particle diameter invalid for this lattice");
            return LBM_ERR_ARG;
        }
        DevParticle d{};
        for (int a = 0; a < 3; ++a) {
            double xa = p.x[a];
            const int Lx = a == 0 ? g.nx : (a == 1 ? g.ny : g.nz);
            if (!(a == 2 && g.bc_z)) {
                xa = std::fmod(xa, (double)Lx);
                if (xa < 0.0) xa += Lx;
            }
            d.x[a] = xa;
            d.u[a] = p.u[a];
            d.w[a] = p.omega[a];
        }
        d.d = p.diameter;
        d.r = 0.5 * p.diameter;
        d.rho = p.density;
        d.fixed = p.fixed ? 1.0 : 0.0;
        up.rec[i] = d;
        maxd = std::max(maxd, p.diameter);
    }
    near_grid(g, maxd, L.box);
    const long long need = near_partial_doubles(L.box, n);
    if ((unsigned long long)need > (unsigned long long)NOALLOC_PARTIAL_DOUBLES) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "request exceeds the fixed scratch: %lld force-partial doubles needed, "
                      "%llu available",
                      need, (unsigned long long)NOALLOC_PARTIAL_DOUBLES);
        set_err(err, err_len, msg);
        return LBM_ERR_ARG;
    }
    const long long mneed = map_entries(g, maxd, n);
    if ((unsigned long long)mneed > (unsigned long long)NOALLOC_MAP_ENTRIES) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "request exceeds the fixed scratch: %lld geometry-map entries needed, "
                      "%llu available",
                      mneed, (unsigned long long)NOALLOC_MAP_ENTRIES);
        set_err(err, err_len, msg);
        return LBM_ERR_ARG;
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        set_err(err, err_len, "no usable current CUDA device");
        return LBM_ERR_CUDA;
    }
    Addresses a;
    if ((e = scratch_addresses(dev, a)) != cudaSuccess) {
        set_err(err, err_len, cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;

    const double lp = -1.0 / cfg->tau;
    const double lm =
        cfg->collision == LBM_TRT ? 1.0 / (cfg->magic / (0.5 + 1.0 / lp) - 0.5) : lp;
    L.kd = make_coll<double>(lp, lm, cfg->rho0, cfg->force_density);
    const bool psm = cfg->coupling <= LBM_PSM_M3B2;
    L.cp.kind = !coupled ? 0 : (psm ? 1 : 2);
    L.cp.variant = psm ? cfg->coupling - LBM_PSM_M1B1 : cfg->coupling - LBM_MEM_BB;
    L.cp.np = n;
    L.cp.subsample = cfg->subsample ? cfg->subsample : 4;
    L.cp.tau = cfg->tau;
    L.cp.rho0 = cfg->rho0;
    L.cp.mr_cpc = L.cp.kind == 2 && L.cp.variant == 2 ? mr_correction_scale(*cfg) : 0.0;
    L.parts = a.particles;
    L.parts_prev = a.particles;
    L.partials = a.partials;
    L.status = status_dev ? status_dev : a.status;
    L.map = a.map;
    region_extent(g, maxd, L.map_ext);
    L.block = dim3(g.tx, g.ty, 1);
    L.stream = s;

    if (!status_dev && (e = cudaMemsetAsync(a.status, 0, sizeof(int), s)) != cudaSuccess) {
        set_err(err, err_len, cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    if (n > 0) {
        // the records travel as a kernel argument, copied at launch: nothing
        // waits for the host array
        k_upload_particles<<<1, MAX_PARTICLES, 0, s>>>(up, n);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_regions(L);
        if (e == cudaSuccess) e = launch_map(L);
    }
    if (e == cudaSuccess) e = launch_bulk(0, src_pdf_dev, dst_pdf_dev, L);
    if (e == cudaSuccess && n > 0) e = launch_near(0, src_pdf_dev, dst_pdf_dev, L);
    if (e == cudaSuccess && n > 0) e = launch_finalize(L, 1, force_torque_dev);
    if (e != cudaSuccess) {
        set_err(err, err_len, cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    set_err(err, err_len, "");
    return LBM_OK;
}
