// C ABI of the coupled D3Q19 library (declarations and contracts in
// include/lbm_gb300.h).  Host orchestration of one global step:
//
//   PSM (Algorithm 2 of Rettinger & Ruede, arXiv:1702.04910):
//     lbm_subcycles (default 1) x bulk + near sweep (solid fractions,
//     weighted collision, force partials) -> averaged force total ->
//     rigid-body update (dt = number of subcycles)
//   MEM (Algorithm 1):
//     lbm_subcycles x (bulk + near sweep with link boundary conditions and
//     link-force partials) -> averaged force total -> rigid-body update
//     (dt = number of subcycles) -> re-mapping with PDF reconstruction
//
// Everything is enqueued on the handle's stream; nothing here synchronises
// except the calls that return data to the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm_gb300.h"
#include "lbm_launch.h"

using namespace lbmgpu;

namespace {

constexpr int N_PROFILE_CLASSES = 6;
enum { PC_BULK = 0, PC_NEAR = 1, PC_FINAL = 2, PC_RIGID = 3, PC_REFILL = 4, PC_OTHER = 5 };

struct EventPair {
    cudaEvent_t a, b;
    int cls;
};

}  // namespace

struct lbm_handle {
    lbm_config cfg;
    cudaStream_t stream;
    cudaStream_t side;           // private stream: near-particle sweep runs beside k_bulk
    cudaEvent_t ev_fork, ev_join;
    int device;
    Geom g;
    int storage;       // 0 FP64, 1 FP32 (PDF storage / arithmetic of every kernel but k_bulk)
    int bulk_mode;     // k_bulk arithmetic: 0 FP64, 1 FP32, 2 float-float, 3 fixed point (FP64 PDFs)
    size_t esize;      // bytes per stored PDF value
    void* buf[2];
    int cur;           // buffer holding the stored state
    int pending_pre;   // buf[cur] holds pre-collision PDFs (first sweep does not stream)
    int kind;          // 0 none, 1 PSM, 2 MEM
    int variant;
    int subcycles;
    int np;
    int have_particles;
    double maxd;
    DevParticle* d_parts;
    DevParticle* d_prev;
    DevParticle* d_tmp;
    double* d_force;     // [np][6]
    double* d_partials;  // [subcycles][np regions][near blocks][np][6]
    size_t partial_cap;  // doubles allocated in d_partials
    unsigned short* d_map;  // per-step geometry map [np][region box]
    size_t map_cap;         // entries allocated in d_map
    int* d_status;
    double* h_stage;     // pinned: status word + np*6 forces
    size_t dev_bytes;
    Coll<double> kd;
    Coll<float> kf;
    Coll<dfloat> kff;
    Coll<fx64> kfx;
    // learned force correction
    lbm_mlp* model;
    int model_mode;    // 0 off, 1 correct, 2 features only
    double u_ref;
    float* d_feat;     // [MAX_PARTICLES][LBM_MLP_IN]
    float* d_corr;     // [MAX_PARTICLES][LBM_MLP_OUT]
    // re-mapping momentum charge (MEM, optional; Algorithm 1 has no such step)
    int remap_charge;
    double* d_charge;       // [np][6] amounts of the last re-mapping, taken off the next step
    double* d_charge_part;  // [np][refill blocks][6] refill-block partials
    size_t charge_part_cap; // doubles allocated in d_charge_part
    // profiling
    int profiling;
    std::vector<EventPair> events;
    std::vector<cudaEvent_t> pool;
    char err[512];
};

namespace {

lbm_status fail(lbm_handle* h, lbm_status st, const char* msg) {
    if (h) std::snprintf(h->err, sizeof(h->err), "%s", msg);
    return st;
}

lbm_status cuda_fail(lbm_handle* h, cudaError_t e, const char* where) {
    if (h)
        std::snprintf(h->err, sizeof(h->err), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define CK(h, call, where)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
    } while (0)

bool is_psm(int c) { return c == LBM_PSM_M1B1 || c == LBM_PSM_M2B2 || c == LBM_PSM_M3B2; }
bool is_mem(int c) { return c == LBM_MEM_BB || c == LBM_MEM_CLI || c == LBM_MEM_MR; }

cudaEvent_t take_event(lbm_handle* h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Records an event before a launch when profiling; returns the pair index.
// The pair is recorded on the stream the kernel is launched on.
int prof_begin(lbm_handle* h, int cls, cudaStream_t s = nullptr) {
    if (!h->profiling) return -1;
    EventPair p{take_event(h), take_event(h), cls};
    if (!p.a || !p.b) return -1;
    cudaEventRecord(p.a, s ? s : h->stream);
    h->events.push_back(p);
    return (int)h->events.size() - 1;
}
void prof_end(lbm_handle* h, int i, cudaStream_t s = nullptr) {
    if (i >= 0) cudaEventRecord(h->events[i].b, s ? s : h->stream);
}

Launch base_launch(lbm_handle* h) {
    Launch L{};
    L.g = h->g;
    L.kd = h->kd;
    L.kf = h->kf;
    L.kff = h->kff;
    L.kfx = h->kfx;
    L.cp.kind = h->kind;
    L.cp.variant = h->variant;
    L.cp.np = h->np;
    L.cp.subsample = h->cfg.subsample;
    L.cp.tau = h->cfg.tau;
    L.cp.rho0 = h->cfg.rho0;
    L.cp.mr_cpc = h->kind == 2 && h->variant == 2 ? mr_correction_scale(h->cfg) : 0.0;
    L.parts = h->d_parts;
    L.parts_prev = h->d_prev;
    L.partials = h->d_partials;
    L.status = h->d_status;
    L.nostream = 0;
    L.all_tiles = 0;
    L.block = dim3(h->g.tx, h->g.ty, 1);
    L.stream = h->stream;
    near_grid(h->g, h->maxd, L.box);
    L.map = h->d_map;
    region_extent(h->g, h->maxd, L.map_ext);
    return L;
}

lbm_status free_particles(lbm_handle* h) {
    cudaFree(h->d_parts);
    cudaFree(h->d_prev);
    cudaFree(h->d_tmp);
    cudaFree(h->d_force);
    cudaFree(h->d_partials);
    cudaFree(h->d_map);
    cudaFree(h->d_charge);
    cudaFree(h->d_charge_part);
    h->d_parts = h->d_prev = h->d_tmp = nullptr;
    h->d_force = h->d_partials = nullptr;
    h->d_map = nullptr;
    h->map_cap = 0;
    h->d_charge = h->d_charge_part = nullptr;
    h->charge_part_cap = 0;
    if (h->h_stage) cudaFreeHost(h->h_stage);
    h->h_stage = nullptr;
    return LBM_OK;
}

lbm_status alloc_particles(lbm_handle* h, int n) {
    free_particles(h);
    size_t np = (size_t)std::max(n, 1);
    size_t part_bytes = sizeof(DevParticle) * np;
    CK(h, cudaMalloc(&h->d_parts, part_bytes), "cudaMalloc particles");
    CK(h, cudaMalloc(&h->d_prev, part_bytes), "cudaMalloc particles");
    CK(h, cudaMalloc(&h->d_tmp, part_bytes), "cudaMalloc particles");
    CK(h, cudaMalloc(&h->d_force, sizeof(double) * 6 * np), "cudaMalloc forces");
    CK(h, cudaMemsetAsync(h->d_force, 0, sizeof(double) * 6 * np, h->stream), "memset");
    CK(h, cudaMalloc(&h->d_charge, sizeof(double) * 6 * np), "cudaMalloc charge");
    CK(h, cudaMemsetAsync(h->d_charge, 0, sizeof(double) * 6 * np, h->stream), "memset");
    CK(h, cudaMallocHost(&h->h_stage, sizeof(double) * (6 * np + 1)), "cudaMallocHost");
    h->partial_cap = 0;
    return LBM_OK;
}

// Force partials for `subcycles` sweeps of the near kernel at the current
// particle count and largest diameter.
lbm_status ensure_partials(lbm_handle* h) {
    int box[3];
    near_grid(h->g, h->maxd, box);
    const size_t need = (size_t)h->subcycles * (size_t)near_partial_doubles(box, h->np);
    const size_t mneed0 = (size_t)map_entries(h->g, h->maxd, h->np);
    if (h->remap_charge) {
        // refill-block partials of the re-mapping charge (box side as in step_once)
        const size_t cneed = (size_t)std::max(h->np, 1) * 6 *
                             (size_t)refill_blocks((int)std::ceil(h->maxd) + 4);
        if (cneed > h->charge_part_cap || !h->d_charge_part) {
            if (h->d_charge_part) {
                CK(h, cudaStreamSynchronize(h->stream), "charge partials sync");
                cudaFree(h->d_charge_part);
                h->d_charge_part = nullptr;
            }
            CK(h, cudaMalloc(&h->d_charge_part, sizeof(double) * cneed),
               "cudaMalloc charge partials");
            h->charge_part_cap = cneed;
        }
    }
    if (need <= h->partial_cap && h->d_partials && mneed0 <= h->map_cap && h->d_map) return LBM_OK;
    if (h->d_partials) {
        CK(h, cudaStreamSynchronize(h->stream), "partials sync");
        cudaFree(h->d_partials);
        h->d_partials = nullptr;
    }
    CK(h, cudaMalloc(&h->d_partials, sizeof(double) * need), "cudaMalloc force partials");
    CK(h, cudaMemsetAsync(h->d_partials, 0, sizeof(double) * need, h->stream), "memset");
    h->partial_cap = need;
    const size_t mneed = (size_t)map_entries(h->g, h->maxd, h->np);
    if (mneed > h->map_cap || !h->d_map) {
        if (h->d_map) cudaFree(h->d_map);
        h->d_map = nullptr;
        CK(h, cudaMalloc(&h->d_map, sizeof(unsigned short) * mneed), "cudaMalloc geometry map");
        CK(h, cudaMemsetAsync(h->d_map, 0, sizeof(unsigned short) * mneed, h->stream), "memset");
        h->map_cap = mneed;
    }
    return LBM_OK;
}

// MEM: collide every cell of the stored pre-collision field (no stream).
lbm_status collide_in_place(lbm_handle* h) {
    Launch L = base_launch(h);
    L.nostream = 1;
    L.all_tiles = 1;
    int pi = prof_begin(h, PC_OTHER);
    CK(h, launch_bulk(h->storage, h->buf[h->cur], h->buf[1 - h->cur], L), "collide launch");
    prof_end(h, pi);
    h->cur = 1 - h->cur;
    h->pending_pre = 0;
    return LBM_OK;
}

// The stored buffer now holds pre-collision PDFs of t = 0.
lbm_status after_pre_state(lbm_handle* h) {
    if (h->kind == 2) return collide_in_place(h);
    h->pending_pre = 1;
    return LBM_OK;
}

// with_map: first sweep of a coupled step; the geometry map of the step's
// particle state is built on the side stream ahead of the near sweep (k_bulk
// does not read it, so it hides under the bulk sweep).
lbm_status sweep(lbm_handle* h, int sub, bool with_map) {
    Launch L = base_launch(h);
    L.nostream = h->pending_pre;
    L.partials = h->d_partials + (size_t)sub * (size_t)near_partial_doubles(L.box, h->np);
    const void* src = h->buf[h->cur];
    void* dst = h->buf[1 - h->cur];
    // The near-particle cells and the bulk cells are disjoint: the (small,
    // latency-bound) near sweep runs on a private stream beside k_bulk.
    if (h->np > 0) {
        CK(h, cudaEventRecord(h->ev_fork, h->stream), "fork record");
        CK(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0), "fork wait");
        Launch Ln = L;
        Ln.stream = h->side;
        if (with_map) {
            int pm = prof_begin(h, PC_OTHER, h->side);
            CK(h, launch_map(Ln), "geometry map launch");
            prof_end(h, pm, h->side);
        }
        int pn = prof_begin(h, PC_NEAR, h->side);
        CK(h, launch_near(h->storage, src, dst, Ln), "near sweep launch");
        prof_end(h, pn, h->side);
        CK(h, cudaEventRecord(h->ev_join, h->side), "join record");
    }
    int pi = prof_begin(h, PC_BULK);
    CK(h, launch_bulk(h->bulk_mode, src, dst, L), "bulk sweep launch");
    prof_end(h, pi);
    if (h->np > 0) CK(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0), "join wait");
    h->cur = 1 - h->cur;
    h->pending_pre = 0;
    return LBM_OK;
}

lbm_status step_once(lbm_handle* h) {
    lbm_status st;
    const int coupled = h->np > 0 && h->kind != 0;
    const int nsub = h->kind != 0 ? h->subcycles : 1;
    // the geometry of the current particle state, shared by the step's
    // sweeps, is built by the first sweep (side stream)
    for (int s = 0; s < nsub; ++s)
        if ((st = sweep(h, s, coupled && s == 0)) != LBM_OK) return st;
    if (!coupled) return LBM_OK;
    Launch L = base_launch(h);
    int pi = prof_begin(h, PC_FINAL);
    CK(h, launch_finalize(L, nsub, h->d_force, h->remap_charge ? h->d_charge : nullptr),
       "force total launch");
    prof_end(h, pi);
    if (h->model_mode) {
        // features of P^n and the flow after the sweeps; corrected force
        pi = prof_begin(h, PC_OTHER);
        CK(h, launch_features(h->storage, h->buf[h->cur], L, h->d_force, h->u_ref, h->d_feat),
           "feature launch");
        if (h->model_mode == 1) {
            // a particle whose features lie beyond 10 standard deviations of
            // the training data keeps the plain force (fallback)
            CK(h, mlp_infer(h->model, h->d_feat, h->np, h->d_corr, 10.0f, h->stream),
               "force model launch");
            CK(h, launch_apply_correction(h->d_corr, h->d_parts, h->np, h->u_ref, h->cfg.rho0,
                                          h->d_force, h->stream),
               "force correction launch");
        }
        prof_end(h, pi);
    }
    pi = prof_begin(h, PC_RIGID);
    CK(h, launch_rigid_body(L, h->d_force, h->cfg.gravity[0], h->cfg.gravity[1],
                            h->cfg.gravity[2], (double)nsub, h->cfg.wall_contact),
       "rigid body launch");
    prof_end(h, pi);
    if (h->kind == 2) {
        // re-map with the new state; rebuild uncovered cells (src of the last sweep)
        L.box[0] = (int)std::ceil(h->maxd) + 4;  // refill: cube side in cells
        pi = prof_begin(h, PC_REFILL);
        CK(h, launch_refill(h->storage, h->buf[1 - h->cur], h->buf[h->cur], L, h->d_prev,
                            h->d_parts, 1, h->remap_charge ? h->d_charge_part : nullptr),
           "refill launch");
        if (h->remap_charge)
            CK(h, launch_charge_total(L, h->d_charge_part, h->d_charge), "charge total launch");
        prof_end(h, pi);
    }
    return LBM_OK;
}

lbm_status read_status(lbm_handle* h) {
    int st = 0;
    CK(h, cudaMemcpyAsync(&h->h_stage[0], h->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                          h->stream),
       "status copy");
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    std::memcpy(&st, &h->h_stage[0], sizeof(int));
    if (st) {
        CK(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream), "status reset");
        // every raised condition is named; the return code follows the first
        // of: domain, index check, instability (particle or fluid), objects
        std::string msg;
        const auto add = [&msg](const char* m) {
            if (!msg.empty()) msg += "; ";
            msg += m;
        };
        if (st & ST_DOMAIN) add("a particle left the domain through a closed wall");
        if (st & ST_BOUNDS) add("an index check in a coupling kernel failed; the step is invalid");
        if (st & ST_FLUID) add("a fluid cell's density became non-finite or <= 0 (the flow is unstable)");
        if (st & ST_UNSTABLE) add("a particle state became non-finite or moved a cell or more per step");
        if (st & ST_TOO_MANY_OBJECTS) add("more than two particles touch one cell");
        const lbm_status code = (st & ST_DOMAIN)                  ? LBM_ERR_DOMAIN
                                : (st & ST_BOUNDS)                ? LBM_ERR_CUDA
                                : (st & (ST_FLUID | ST_UNSTABLE)) ? LBM_ERR_UNSTABLE
                                : (st & ST_TOO_MANY_OBJECTS)      ? LBM_ERR_UNSUPPORTED
                                                                  : LBM_ERR_CUDA;
        if (!msg.empty()) return fail(h, code, msg.c_str());
        return fail(h, LBM_ERR_CUDA, "device status raised");
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_abi_version(void) { return 1; }

const char* lbm_last_error(const lbm_handle* h) {
    return h ? h->err : "no handle";
}

size_t lbm_device_bytes(const lbm_handle* h) {
    if (!h) return 0;
    const size_t np = (size_t)std::max(h->np, 1);
    return h->dev_bytes + 3 * sizeof(DevParticle) * np + sizeof(double) * 6 * np +
           sizeof(double) * h->partial_cap + sizeof(unsigned short) * h->map_cap +
           sizeof(double) * 6 * np + sizeof(double) * h->charge_part_cap;
}

lbm_status lbm_create(const lbm_config* cfg, void* stream, lbm_handle** out) {
    if (!cfg || !out) return LBM_ERR_ARG;
    *out = nullptr;
    {
        const lbm_status st = check_config(*cfg);
        if (st != LBM_OK) return st;
    }
    const long long n = (long long)cfg->nx * cfg->ny * cfg->nz;

    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return LBM_ERR_OOM;
    h->cfg = *cfg;
    if (h->cfg.subsample == 0) h->cfg.subsample = 4;
    h->stream = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    {
        // the near sweep's stream has the highest priority: its few long-lived
        // blocks are placed as soon as k_bulk blocks retire, instead of
        // waiting behind the whole bulk grid
        int lo_prio = 0, hi_prio = 0;
        cudaError_t e0 = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
        if (e0 == cudaSuccess) e0 = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi_prio);
        if (e0 == cudaSuccess) e0 = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e0 == cudaSuccess) e0 = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        if (e0 != cudaSuccess) {
            lbm_status st0 = cuda_fail(h, e0, "stream / event creation");
            lbm_destroy(h);
            return st0;
        }
    }
    // kernel storage codes: 0 FP64, 1 FP32, 4 FP16 shifted, 5 BF16 shifted
    h->storage = cfg->storage == LBM_STORE_F32     ? 1
                 : cfg->storage == LBM_STORE_F16S  ? 4
                 : cfg->storage == LBM_STORE_BF16S ? 5
                                                   : 0;
    h->esize = h->storage == 0 ? sizeof(double) : (h->storage == 1 ? sizeof(float) : 2);
    h->bulk_mode = cfg->storage;  // bulk arithmetic: the storage code, or 2 / 3 on FP64 state
    h->kind = is_psm(cfg->coupling) ? 1 : (is_mem(cfg->coupling) ? 2 : 0);
    h->variant = h->kind == 1 ? cfg->coupling - LBM_PSM_M1B1
                              : (h->kind == 2 ? cfg->coupling - LBM_MEM_BB : 0);
    // MEM: 2 sweeps by default (Algorithm 1); PSM: 1 (Algorithm 2), or the
    // two averaged subcycles of the settling benchmark of Sec. 4.1 on request
    h->subcycles = cfg->lbm_subcycles > 0 ? cfg->lbm_subcycles : (h->kind == 2 ? 2 : 1);
    if (h->kind == 0) h->subcycles = 1;

    Geom& g = h->g;
    g.nx = cfg->nx;
    g.ny = cfg->ny;
    g.nz = cfg->nz;
    g.bc_z = cfg->bc_z;
    g.n = n;
    set_open_boundaries(g, *cfg);
    g.tx = cfg->nx >= 128 ? 128 : (cfg->nx >= 64 ? 64 : 32);
    g.ty = 256 / g.tx;
    g.ntx = (cfg->nx + g.tx - 1) / g.tx;
    g.nty = (cfg->ny + g.ty - 1) / g.ty;
    g.tz = cfg->storage == LBM_STORE_F32 ? 2 : 1;  // two z cells per thread (k_bulk)
    g.ntz = (cfg->nz + g.tz - 1) / g.tz;

    const double lp = -1.0 / cfg->tau;
    const double lm = cfg->collision == LBM_TRT ? 1.0 / (cfg->magic / (0.5 + 1.0 / lp) - 0.5) : lp;
    h->kd = make_coll<double>(lp, lm, cfg->rho0, cfg->force_density);
    h->kf = make_coll<float>(lp, lm, cfg->rho0, cfg->force_density);
    h->kff = make_coll<dfloat>(lp, lm, cfg->rho0, cfg->force_density);
    h->kfx = make_coll<fx64>(lp, lm, cfg->rho0, cfg->force_density);

    size_t bytes = (size_t)NQ * (size_t)n * h->esize;
    cudaError_t e = cudaMalloc(&h->buf[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->buf[1], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(int));
    if (e != cudaSuccess) {
        lbm_status st = cuda_fail(h, e, "cudaMalloc PDF buffers");
        lbm_destroy(h);
        return st;
    }
    h->dev_bytes = 2 * bytes + sizeof(int);
    cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream);
    lbm_status st = alloc_particles(h, 0);
    if (st == LBM_OK) st = ensure_partials(h);
    if (st == LBM_OK) {
        const double u0[3] = {0.0, 0.0, 0.0};
        st = lbm_init_equilibrium(h, cfg->rho0, u0);
    }
    if (st != LBM_OK) {
        lbm_destroy(h);
        return st;
    }
    *out = h;
    return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
    cudaFree(h->d_status);
    cudaFree(h->d_feat);
    cudaFree(h->d_corr);
    free_particles(h);
    for (auto& p : h->events) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
    delete h;
}

lbm_status lbm_set_particles(lbm_handle* h, int n, const lbm_particle* host_in) {
    if (!h) return LBM_ERR_ARG;
    if (n < 0 || n > MAX_PARTICLES || (n > 0 && !host_in))
        return fail(h, LBM_ERR_ARG, "particle count must be 0..32");
    double maxd = 0.0;
    for (int i = 0; i < n; ++i) {
        const lbm_particle& p = host_in[i];
        const double D = p.diameter;
        bool finite = std::isfinite(D) && std::isfinite(p.density);
        for (int a = 0; a < 3; ++a)
            finite = finite && std::isfinite(p.x[a]) && std::isfinite(p.u[a]) && std::isfinite(p.omega[a]);
        if (!finite || !(D >= 1.0) || !(p.density > 0.0))
            return fail(h, LBM_ERR_ARG, "particle with non-finite value, D < 1 or density <= 0");
        const double need = D + 2.0 * NEAR_HALO + 2.0;
        if (need > h->g.nx || need > h->g.ny || (!h->g.bc_z && need > h->g.nz))
            return fail(h, LBM_ERR_ARG, "particle diameter + 6 exceeds a periodic extent");
        const double margin = h->g.bc_z == 2 ? OPEN_MARGIN : 0.0;
        if (h->g.bc_z && (p.x[2] - 0.5 * D - margin < 0.0 || p.x[2] + 0.5 * D + margin > h->g.nz))
            return fail(h, LBM_ERR_ARG,
                        "particle crosses a closed wall or comes within R + 3 of an open boundary");
        maxd = std::max(maxd, D);
    }
    const bool remap = h->have_particles && h->kind == 2 && n == h->np && n > 0;
    if (h->have_particles && h->kind == 2 && n != h->np && h->np > 0)
        return fail(h, LBM_ERR_ARG, "the particle count cannot change once MEM particles are mapped");
    std::vector<DevParticle> recs((size_t)std::max(n, 1));
    for (int i = 0; i < n; ++i) {
        const lbm_particle& p = host_in[i];
        DevParticle d{};
        for (int a = 0; a < 3; ++a) {
            double xa = p.x[a];
            const int L = a == 0 ? h->g.nx : (a == 1 ? h->g.ny : h->g.nz);
            if (!(a == 2 && h->g.bc_z)) {
                xa = std::fmod(xa, (double)L);
                if (xa < 0.0) xa += L;
            }
            d.x[a] = xa;
            d.u[a] = p.u[a];
            d.w[a] = p.omega[a];
        }
        d.d = p.diameter;
        d.r = 0.5 * p.diameter;
        d.rho = p.density;
        d.fixed = p.fixed ? 1.0 : 0.0;
        recs[i] = d;
    }
    if (n != h->np || !h->d_parts) {
        h->np = n;
        lbm_status st = alloc_particles(h, n);
        if (st != LBM_OK) return st;
    }
    // a replacement from the host clears the pending re-mapping charge
    CK(h, cudaMemsetAsync(h->d_charge, 0, sizeof(double) * 6 * (size_t)std::max(n, 1), h->stream),
       "charge reset");
    h->maxd = std::max(h->maxd, maxd);
    {
        lbm_status st = ensure_partials(h);
        if (st != LBM_OK) return st;
    }
    if (remap)
        CK(h, cudaMemcpyAsync(h->d_tmp, h->d_parts, sizeof(DevParticle) * n,
                              cudaMemcpyDeviceToDevice, h->stream),
           "particle copy");
    if (n > 0) {
        CK(h, cudaMemcpyAsync(h->d_parts, recs.data(), sizeof(DevParticle) * n,
                              cudaMemcpyHostToDevice, h->stream),
           "particle upload");
        CK(h, cudaMemcpyAsync(h->d_prev, recs.data(), sizeof(DevParticle) * n,
                              cudaMemcpyHostToDevice, h->stream),
           "particle upload");
    }
    CK(h, cudaStreamSynchronize(h->stream), "particle upload sync");  // recs is pageable
    Launch L = base_launch(h);
    CK(h, launch_regions(L), "region launch");
    L.parts = h->d_prev;
    CK(h, launch_regions(L), "region launch");
    if (remap) {
        L = base_launch(h);
        L.box[0] = (int)std::ceil(h->maxd) + 4;
        CK(h, launch_refill(h->storage, h->buf[1 - h->cur], h->buf[h->cur], L, h->d_tmp, h->d_parts, 0),
           "refill launch");
    }
    h->have_particles = n > 0;
    return LBM_OK;
}

lbm_status lbm_get_particles(lbm_handle* h, lbm_particle* host_out) {
    if (!h) return LBM_ERR_ARG;
    if (h->np == 0) return read_status(h);
    if (!host_out) return fail(h, LBM_ERR_ARG, "null output");
    std::vector<DevParticle> recs((size_t)h->np);
    CK(h, cudaMemcpyAsync(recs.data(), h->d_parts, sizeof(DevParticle) * h->np,
                          cudaMemcpyDeviceToHost, h->stream),
       "particle download");
    lbm_status st = read_status(h);
    for (int i = 0; i < h->np; ++i) {
        lbm_particle& p = host_out[i];
        for (int a = 0; a < 3; ++a) {
            p.x[a] = recs[i].x[a];
            p.u[a] = recs[i].u[a];
            p.omega[a] = recs[i].w[a];
        }
        p.diameter = recs[i].d;
        p.density = recs[i].rho;
        p.fixed = recs[i].fixed != 0.0;
    }
    return st;
}

lbm_status lbm_init_equilibrium(lbm_handle* h, double rho, const double u[3]) {
    if (!h || !u) return LBM_ERR_ARG;
    if (!std::isfinite(rho) || !std::isfinite(u[0]) || !std::isfinite(u[1]) || !std::isfinite(u[2]))
        return fail(h, LBM_ERR_ARG, "non-finite initial state");
    Launch L = base_launch(h);
    CK(h, launch_init_eq(h->storage, h->buf[h->cur], L, rho, u[0], u[1], u[2]), "init launch");
    return after_pre_state(h);
}

lbm_status lbm_step(lbm_handle* h, int nsteps) {
    if (!h || nsteps < 0) return LBM_ERR_ARG;
    for (int i = 0; i < nsteps; ++i) {
        lbm_status st = step_once(h);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

lbm_status lbm_get_forces(lbm_handle* h, double* F, double* T) {
    if (!h) return LBM_ERR_ARG;
    if (h->np == 0) return read_status(h);
    if (!F || !T) return fail(h, LBM_ERR_ARG, "null output");
    CK(h, cudaMemcpyAsync(h->h_stage + 1, h->d_force, sizeof(double) * 6 * h->np,
                          cudaMemcpyDeviceToHost, h->stream),
       "force download");
    lbm_status st = read_status(h);
    for (int i = 0; i < h->np; ++i)
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] = h->h_stage[1 + 6 * i + a];
            T[3 * i + a] = h->h_stage[1 + 6 * i + 3 + a];
        }
    return st;
}

lbm_status lbm_set_remap_charge(lbm_handle* h, int enable) {
    if (!h || (enable != 0 && enable != 1)) return LBM_ERR_ARG;
    if (enable && h->kind != 2)
        return fail(h, LBM_ERR_UNSUPPORTED, "the re-mapping momentum charge applies to MEM couplings");
    h->remap_charge = enable;
    if (h->d_charge)
        CK(h, cudaMemsetAsync(h->d_charge, 0, sizeof(double) * 6 * (size_t)std::max(h->np, 1),
                              h->stream),
           "charge reset");
    if (enable && h->have_particles) return ensure_partials(h);
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_handle* h, int what, void* dst, size_t bytes, int dst_is_device) {
    if (!h || !dst) return LBM_ERR_ARG;
    const size_t n = (size_t)h->g.n;
    size_t need;
    switch (what) {
        case LBM_FIELD_PDF: need = (size_t)NQ * n * h->esize; break;
        case LBM_FIELD_RHO:
        case LBM_FIELD_EPS: need = n * sizeof(double); break;
        case LBM_FIELD_U: need = 3 * n * sizeof(double); break;
        case LBM_FIELD_FLAG: need = n * sizeof(int); break;
        case LBM_FIELD_PDF_F64: need = (size_t)NQ * n * sizeof(double); break;
        case LBM_FIELD_REMAP_CHARGE: need = (size_t)6 * h->np * sizeof(double); break;
        default: return fail(h, LBM_ERR_ARG, "unknown field");
    }
    if (bytes != need) return fail(h, LBM_ERR_ARG, "byte count does not match the field");
    if (what == LBM_FIELD_REMAP_CHARGE) {
        if (need > 0)
            CK(h, cudaMemcpyAsync(dst, h->d_charge, need,
                                  dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  h->stream),
               "charge copy");
        return read_status(h);
    }
    if (what == LBM_FIELD_PDF) {
        CK(h, cudaMemcpyAsync(dst, h->buf[h->cur], need,
                              dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              h->stream),
           "field copy");
        return read_status(h);
    }
    void* out = dst;
    if (!dst_is_device) CK(h, cudaMalloc(&out, need), "cudaMalloc field");
    Launch L = base_launch(h);
    L.nostream = h->pending_pre;
    cudaError_t e = what == LBM_FIELD_PDF_F64
                        ? launch_to_f64(h->storage, h->buf[h->cur], (double*)out,
                                        (long long)NQ * (long long)n, (long long)n, h->stream)
                        : launch_macro(h->storage, h->buf[h->cur], L, what, out);
    if (e == cudaSuccess && !dst_is_device)
        e = cudaMemcpyAsync(dst, out, need, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (!dst_is_device) cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(h, e, "field kernel");
    return read_status(h);
}

lbm_status lbm_set_fields(lbm_handle* h, int what, const void* src, size_t bytes, int src_is_device) {
    if (!h || !src) return LBM_ERR_ARG;
    const size_t n = (size_t)h->g.n;
    if (what == LBM_FIELD_REMAP_CHARGE) {
        const size_t need = (size_t)6 * h->np * sizeof(double);
        if (bytes != need) return fail(h, LBM_ERR_ARG, "byte count does not match the field");
        if (need > 0) {
            CK(h, cudaMemcpyAsync(h->d_charge, src, need,
                                  src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  h->stream),
               "charge copy");
            CK(h, cudaStreamSynchronize(h->stream), "charge copy sync");
        }
        return LBM_OK;
    }
    if (what == LBM_FIELD_PDF) {
        const size_t need = (size_t)NQ * n * h->esize;
        if (bytes != need) return fail(h, LBM_ERR_ARG, "byte count does not match the field");
        CK(h, cudaMemcpyAsync(h->buf[h->cur], src, need,
                              src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              h->stream),
           "field copy");
        CK(h, cudaStreamSynchronize(h->stream), "field copy sync");
        h->pending_pre = 0;
        return LBM_OK;
    }
    if (what == LBM_FIELD_PDF_PRE) {
        const size_t need = (size_t)NQ * n * sizeof(double);
        if (bytes != need) return fail(h, LBM_ERR_ARG, "byte count does not match the field");
        const double* dsrc = (const double*)src;
        double* tmp = nullptr;
        if (!src_is_device) {
            CK(h, cudaMalloc(&tmp, need), "cudaMalloc staging");
            cudaError_t e = cudaMemcpyAsync(tmp, src, need, cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) {
                cudaFree(tmp);
                return cuda_fail(h, e, "field upload");
            }
            dsrc = tmp;
        }
        cudaError_t e = launch_from_f64(h->storage, dsrc, h->buf[h->cur],
                                        (long long)NQ * (long long)n, (long long)n, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (tmp) cudaFree(tmp);
        if (e != cudaSuccess) return cuda_fail(h, e, "field conversion");
        return after_pre_state(h);
    }
    return fail(h, LBM_ERR_ARG, "field cannot be set");
}

lbm_status lbm_synchronize(lbm_handle* h) {
    if (!h) return LBM_ERR_ARG;
    return read_status(h);
}

lbm_status lbm_set_force_model(lbm_handle* h, lbm_mlp* m, double u_ref, int mode) {
    if (!h) return LBM_ERR_ARG;
    if (mode < 0 || mode > 2 || (mode == 1 && !m) || (mode != 0 && !(u_ref > 0.0)))
        return fail(h, LBM_ERR_ARG, "mode 0..2; mode 1 needs a model; u_ref > 0");
    if (mode && h->kind == 0) return fail(h, LBM_ERR_ARG, "a force model needs a coupling");
    if (mode && !h->d_feat) {
        CK(h, cudaMalloc(&h->d_feat, sizeof(float) * MAX_PARTICLES * LBM_MLP_IN), "cudaMalloc features");
        CK(h, cudaMalloc(&h->d_corr, sizeof(float) * MAX_PARTICLES * LBM_MLP_OUT), "cudaMalloc features");
        CK(h, cudaMemsetAsync(h->d_feat, 0, sizeof(float) * MAX_PARTICLES * LBM_MLP_IN, h->stream),
           "memset");
    }
    h->model = mode == 1 ? m : nullptr;
    h->model_mode = mode;
    h->u_ref = u_ref;
    return LBM_OK;
}

lbm_status lbm_get_features(lbm_handle* h, float* host, size_t count) {
    if (!h || !host) return LBM_ERR_ARG;
    if (!h->d_feat) return fail(h, LBM_ERR_ARG, "no force model attached");
    if (count != (size_t)h->np * LBM_MLP_IN) return fail(h, LBM_ERR_ARG, "count must be np * LBM_MLP_IN");
    if (count == 0) return read_status(h);
    CK(h, cudaMemcpyAsync(host, h->d_feat, sizeof(float) * count, cudaMemcpyDeviceToHost, h->stream),
       "feature download");
    return read_status(h);
}

lbm_status lbm_profile_enable(lbm_handle* h, int enable) {
    if (!h) return LBM_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream), "profile sync");
    for (auto& p : h->events) {
        h->pool.push_back(p.a);
        h->pool.push_back(p.b);
    }
    h->events.clear();
    h->profiling = enable ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_profile_read(lbm_handle* h, int n_classes, double* ms, long long* launches) {
    if (!h || n_classes < 0 || (n_classes > 0 && (!ms || !launches))) return LBM_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream), "profile sync");
    for (int k = 0; k < n_classes; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (auto& p : h->events) {
        float t = 0.0f;
        CK(h, cudaEventElapsedTime(&t, p.a, p.b), "event elapsed");
        if (p.cls < n_classes) {
            ms[p.cls] += t;
            launches[p.cls] += 1;
        }
    }
    return LBM_OK;
}

}  // extern "C"
