// Batched ensemble of independent single-sphere cases (declarations and
// contracts in include/lbm_gb300.h).
//
// Layout in HBM: one allocation (the arena) holds, in 256-byte aligned
// slices, the case records, the status word, the particle records (current
// and previous state of every case, contiguous), the forces [case][6], the
// work lists, and per case its two PDF buffers (SoA, 19 x N doubles each),
// its force partials (subcycles x near blocks x 6) and its geometry map.
//
// One global step is captured once as a CUDA graph on a private stream:
//
//   for s < max subcycles:   [s = 0: map (all cases)] -> near (cases with
//                            > s sweeps, side branch)
//                            || bulk (same cases, persistent)  -> swap
//   force total -> rigid-body update (all cases) -> refill (MEM cases)
//
// and lbm_batch_step replays it on the batch's stream.  Each case's kernels
// read buf[cur] and write buf[1 - cur]; the swap kernel flips cur on the
// device, so every replay is the same graph.
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

constexpr int MAX_CASES = 4096;
thread_local char g_create_err[512];  // why the last lbm_batch_create on this thread failed

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Device work list of one launch: cases and prefix sums of their items.
struct WorkList {
    int* list = nullptr;
    long long* base = nullptr;
    int n = 0;
    long long total = 0;
    std::vector<int> h_list;
    std::vector<long long> h_base;
    BatchList view() const { return BatchList{list, base, n}; }
};

}  // namespace

struct lbm_batch {
    int n;
    int mode;  // bulk collision arithmetic: 0 FP64, 3 fixed point
    cudaStream_t stream;
    cudaStream_t cap, side;
    cudaEvent_t ev_fork, ev_join, t0, t1;
    std::vector<lbm_config> cfg;
    std::vector<BatchCase> hc;
    int max_sub;
    int any_mem;
    void* arena;
    size_t arena_bytes;
    BatchCase* dcases;
    int* dstatus;
    DevParticle* dparts;
    DevParticle* dprev;
    double* dforce;
    WorkList map_l, refill_l;
    std::vector<WorkList> near_l, bulk_l;  // per subcycle
    WorkList one;              // single-case list used by the autotuner
    std::vector<int> layouts;  // bulk tiling of each case (LBM_BATCH_*)
    int grid;
    int resident;  // resident bulk blocks on the GPU (SMs x blocks per SM)
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int graph_kernels;
    long long cell_updates;
    int profiling;                 // the graph brackets each bulk sweep with stamps
    int any_charge;                // a MEM case charges its re-mapping momentum
    unsigned long long* dprof;     // [start, summed ns, launches]
    char err[512];
};

namespace {

lbm_status fail(lbm_batch* b, lbm_status st, const char* msg) {
    if (b) std::snprintf(b->err, sizeof(b->err), "%s", msg);
    return st;
}

lbm_status cuda_fail(lbm_batch* b, cudaError_t e, const char* where) {
    if (b)
        std::snprintf(b->err, sizeof(b->err), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define BK(b, call, where)                                      \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(b, e_, where);  \
    } while (0)

int layout_tx(int layout) { return layout == LBM_BATCH_BOX64 ? 64 : (layout == LBM_BATCH_BOX128 ? 128 : 32); }

// Box tiling of a case's lattice for a layout (the plane layout keeps the
// 32-wide box fields; its kernel does not use them).
void set_tiling(Geom& g, int layout) {
    g.tx = layout_tx(layout);
    g.ty = 256 / g.tx;
    g.ntx = (g.nx + g.tx - 1) / g.tx;
    g.nty = (g.ny + g.ty - 1) / g.ty;
    g.tz = 1;
    g.ntz = g.nz;
}

long long bulk_items(const Geom& g, int layout) {
    if (layout == LBM_BATCH_PLANE) return (long long)((g.nx * g.ny + 255) / 256) * g.nz;
    return (long long)g.ntx * g.nty * g.ntz;
}

long long map_items(const BatchCase& c) {
    return (long long)((c.map_ext[0] + 31) / 32) * c.map_ext[1] * c.map_ext[2];
}

long long refill_items(const BatchCase& c) {
    const long long s = c.refill_side;
    return (s * s * s + REFILL_THREADS - 1) / REFILL_THREADS;
}

void fill_list(WorkList& w, const std::vector<int>& cases, const std::vector<long long>& items) {
    w.n = (int)cases.size();
    w.h_list = cases;
    w.h_base.assign(cases.size() + 1, 0);
    for (size_t i = 0; i < cases.size(); ++i) w.h_base[i + 1] = w.h_base[i] + items[i];
    w.total = w.h_base.back();
}

lbm_status upload_list(lbm_batch* b, WorkList& w) {
    if (w.n == 0) return LBM_OK;
    BK(b, cudaMemcpyAsync(w.list, w.h_list.data(), sizeof(int) * w.n, cudaMemcpyHostToDevice,
                          b->stream),
       "work list upload");
    BK(b, cudaMemcpyAsync(w.base, w.h_base.data(), sizeof(long long) * (w.n + 1),
                          cudaMemcpyHostToDevice, b->stream),
       "work list upload");
    return LBM_OK;
}

// Applies per-case bulk layouts: re-tiles every case, recomputes the
// particle regions' tile ranges and the bulk work lists.  Synchronises.
lbm_status apply_layouts(lbm_batch* b, const std::vector<int>& lays) {
    for (int i = 0; i < b->n; ++i) {
        BatchCase& c = b->hc[i];
        set_tiling(c.g, lays[i]);
        c.layout = lays[i] == LBM_BATCH_PLANE ? 1 : 0;
        // cur lives on the device and is flipped there: write only the tiling
        BK(b, cudaMemcpyAsync(&b->dcases[i].g, &c.g, sizeof(Geom), cudaMemcpyHostToDevice,
                              b->stream),
           "case upload");
        BK(b, cudaMemcpyAsync(&b->dcases[i].layout, &c.layout, sizeof(int), cudaMemcpyHostToDevice,
                              b->stream),
           "case upload");
    }
    BK(b, launch_batch_regions(b->dcases, b->n, b->stream), "region launch");
    for (int s = 0; s < b->max_sub; ++s) {
        std::vector<long long> items;
        for (int c : b->bulk_l[s].h_list) items.push_back(bulk_items(b->hc[c].g, lays[c]));
        std::vector<int> cases = b->bulk_l[s].h_list;
        fill_list(b->bulk_l[s], cases, items);
        lbm_status st = upload_list(b, b->bulk_l[s]);
        if (st != LBM_OK) return st;
    }
    BK(b, cudaStreamSynchronize(b->stream), "layout sync");  // host vectors above are pageable
    b->layouts = lays;
    return LBM_OK;
}

void destroy_graph(lbm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Enqueues one global step on the capture stream (see the file comment).
cudaError_t enqueue_step(lbm_batch* b, int* kernels) {
    cudaStream_t s = b->cap;
    int k = 0;
    cudaError_t e = cudaSuccess;
    for (int sub = 0; sub < b->max_sub && e == cudaSuccess; ++sub) {
        const WorkList& nl = b->near_l[sub];
        const WorkList& bl = b->bulk_l[sub];
        // near-particle and bulk cells are disjoint: the near sweep is a
        // parallel branch of the graph; the first one builds the step's
        // geometry map first (the bulk sweep does not read it)
        e = cudaEventRecord(b->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->ev_fork, 0);
        if (e == cudaSuccess && sub == 0) {
            e = launch_batch_map(b->dcases, b->map_l.view(), b->map_l.total, b->side);
            ++k;
        }
        if (e == cudaSuccess) e = launch_batch_near(b->dcases, nl.view(), nl.total, sub, b->dstatus, b->side);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_join, b->side);
        if (e == cudaSuccess && b->profiling) {
            e = launch_stamp(b->dprof, 0, s);
            ++k;
        }
        if (e == cudaSuccess) e = launch_batch_bulk(b->mode, b->dcases, bl.view(), bl.total, b->grid, b->dstatus, s);
        if (e == cudaSuccess && b->profiling) {
            e = launch_stamp(b->dprof, 1, s);
            ++k;
        }
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join, 0);
        if (e == cudaSuccess) e = launch_batch_swap(b->dcases, nl.view(), s);
        k += 3;
    }
    if (e == cudaSuccess) e = launch_batch_finalize(b->dcases, b->n, s);
    if (e == cudaSuccess) e = launch_batch_rigid(b->dcases, b->n, b->dstatus, s);
    k += 2;
    if (e == cudaSuccess && b->refill_l.n > 0) {
        e = launch_batch_refill(b->dcases, b->refill_l.view(), b->refill_l.total, b->dstatus, s);
        ++k;
        if (e == cudaSuccess && b->any_charge) {
            e = launch_batch_charge_total(b->dcases, b->n, s);
            ++k;
        }
    }
    *kernels = k;
    return e;
}

lbm_status build_graph(lbm_batch* b) {
    destroy_graph(b);
    BK(b, cudaStreamSynchronize(b->stream), "graph sync");
    BK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    int kernels = 0;
    cudaError_t e = enqueue_step(b, &kernels);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(b, e, "step capture");
    }
    b->graph = g;
    BK(b, cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
    b->graph_kernels = kernels;
    return LBM_OK;
}

lbm_status read_status(lbm_batch* b) {
    int st = 0;
    BK(b, cudaMemcpyAsync(&st, b->dstatus, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
       "status copy");
    BK(b, cudaStreamSynchronize(b->stream), "stream synchronize");
    if (st) {
        BK(b, cudaMemsetAsync(b->dstatus, 0, sizeof(int), b->stream), "status reset");
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
        if (!msg.empty()) return fail(b, code, msg.c_str());
        return fail(b, LBM_ERR_CUDA, "device status raised");
    }
    return LBM_OK;
}

// Validates case c; fills its record except for the device pointers.
lbm_status make_case(lbm_batch* b, int c, const lbm_config& cfg, const lbm_particle& p,
                     int storage, BatchCase& out, DevParticle& rec) {
    char msg[200];
    auto bad = [&](const char* why) {
        std::snprintf(msg, sizeof(msg), "case %d: %s", c, why);
        return fail(b, LBM_ERR_ARG, msg);
    };
    if (cfg.nx < 1 || cfg.ny < 1 || cfg.nz < 1) return bad("lattice extent < 1");
    if ((long long)cfg.nx * cfg.ny > (1LL << 30) || (long long)cfg.nx * cfg.ny * cfg.nz > (1LL << 36))
        return bad("lattice too large");
    if (!(cfg.tau > 0.5) || !std::isfinite(cfg.tau) || !(cfg.rho0 > 0.0) || !std::isfinite(cfg.rho0))
        return bad("tau <= 1/2 or rho0 <= 0");
    if (cfg.collision != LBM_BGK && cfg.collision != LBM_TRT) return bad("unknown collision");
    if (cfg.bc_z != 0 && cfg.bc_z != 1) return bad("bc_z must be 0 or 1");
    if (cfg.subsample < 0 || cfg.subsample > 40 || cfg.lbm_subcycles < 0 || cfg.lbm_subcycles > 16)
        return bad("subsample or subcycles out of range");
    if (cfg.coupling < LBM_PSM_M1B1 || cfg.coupling > LBM_MEM_MR)
        return bad("coupling must be a PSM or MEM variant");
    if (cfg.coupling == LBM_MEM_MR && !mr_supported(cfg)) {
        std::snprintf(msg, sizeof(msg), "case %d: MEM MR needs |Lambda_- - 1/2| >= 0.01", c);
        return fail(b, LBM_ERR_UNSUPPORTED, msg);
    }
    if (cfg.storage != storage) return bad("storage differs from case 0");
    double lp = -1.0 / cfg.tau, lm = lp;
    if (cfg.collision == LBM_TRT) {
        const double denom = cfg.magic / (0.5 + 1.0 / lp) - 0.5;
        if (!(cfg.magic > 0.0) || denom == 0.0) return bad("invalid TRT magic parameter");
        lm = 1.0 / denom;
        if (!(lm > -2.0 && lm < 0.0)) return bad("TRT lambda- out of (-2, 0)");
    }
    bool finite = std::isfinite(p.diameter) && std::isfinite(p.density);
    for (int a = 0; a < 3; ++a)
        finite = finite && std::isfinite(p.x[a]) && std::isfinite(p.u[a]) && std::isfinite(p.omega[a]) &&
                 std::isfinite(cfg.gravity[a]) && std::isfinite(cfg.force_density[a]);
    if (!finite || !(p.diameter >= 1.0) || !(p.density > 0.0))
        return bad("particle with non-finite value, D < 1 or density <= 0");
    const double need = p.diameter + 2.0 * NEAR_HALO + 2.0;
    if (need > cfg.nx || need > cfg.ny || (!cfg.bc_z && need > cfg.nz))
        return bad("particle diameter + 6 exceeds a periodic extent");
    if (cfg.bc_z && (p.x[2] - 0.5 * p.diameter < 0.0 || p.x[2] + 0.5 * p.diameter > cfg.nz))
        return bad("particle crosses a closed wall");

    BatchCase k{};
    Geom& g = k.g;
    g.nx = cfg.nx;
    g.ny = cfg.ny;
    g.nz = cfg.nz;
    g.bc_z = cfg.bc_z;
    g.n = (long long)cfg.nx * cfg.ny * cfg.nz;
    set_open_boundaries(g, cfg);
    set_tiling(g, LBM_BATCH_PLANE);
    const bool psm = cfg.coupling <= LBM_PSM_M3B2;
    k.kind = psm ? 1 : 2;
    k.subcycles = cfg.lbm_subcycles > 0 ? cfg.lbm_subcycles : (psm ? 1 : 2);
    k.wall_contact = cfg.wall_contact ? 1 : 0;
    k.cp.kind = k.kind;
    k.cp.variant = psm ? cfg.coupling - LBM_PSM_M1B1 : cfg.coupling - LBM_MEM_BB;
    k.cp.np = 1;
    k.cp.subsample = cfg.subsample ? cfg.subsample : 4;
    k.cp.tau = cfg.tau;
    k.cp.rho0 = cfg.rho0;
    k.cp.mr_cpc = cfg.coupling == LBM_MEM_MR ? mr_correction_scale(cfg) : 0.0;
    k.kd = make_coll<double>(lp, lm, cfg.rho0, cfg.force_density);
    k.kfx = make_coll<fx64>(lp, lm, cfg.rho0, cfg.force_density);
    region_extent(g, p.diameter, k.map_ext);
    near_grid(g, p.diameter, k.box);
    k.nblk = near_blocks(k.box);
    k.refill_side = (int)std::ceil(p.diameter) + 4;
    for (int a = 0; a < 3; ++a) k.gravity[a] = cfg.gravity[a];
    k.cur = 0;

    DevParticle d{};
    for (int a = 0; a < 3; ++a) {
        double xa = p.x[a];
        const int L = a == 0 ? g.nx : (a == 1 ? g.ny : g.nz);
        if (!(a == 2 && g.bc_z)) {
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
    out = k;
    rec = d;
    return LBM_OK;
}

void release(lbm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    destroy_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    if (b->dprof) cudaFree(b->dprof);
    if (b->arena) cudaFree(b->arena);
    delete b;
}

// Mean duration (ms) of `reps` launches of the bulk kernel over list w at
// the given grid.  src = buf[cur], dst = buf[1 - cur]: the next sweep
// overwrites every cell this writes, so the simulation state is unchanged.
lbm_status time_bulk(lbm_batch* b, const WorkList& w, int grid, int reps, double* ms) {
    BK(b, launch_batch_bulk(b->mode, b->dcases, w.view(), w.total, grid, b->dstatus, b->stream), "tuning launch");
    BK(b, cudaEventRecord(b->t0, b->stream), "event record");
    for (int r = 0; r < reps; ++r)
        BK(b, launch_batch_bulk(b->mode, b->dcases, w.view(), w.total, grid, b->dstatus, b->stream),
           "tuning launch");
    BK(b, cudaEventRecord(b->t1, b->stream), "event record");
    BK(b, cudaEventSynchronize(b->t1), "event sync");
    float t = 0.0f;
    BK(b, cudaEventElapsedTime(&t, b->t0, b->t1), "event elapsed");
    *ms = (double)t / reps;
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(int n_cases, const lbm_config* cfgs, const lbm_particle* particles,
                            void* stream, lbm_batch** out) {
    g_create_err[0] = 0;
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (n_cases < 1 || n_cases > MAX_CASES || !cfgs || !particles) {
        std::snprintf(g_create_err, sizeof(g_create_err), "n_cases must be 1..%d with configs and particles", MAX_CASES);
        return LBM_ERR_ARG;
    }
    const int storage = cfgs[0].storage;
    if (storage != LBM_STORE_F64 && storage != LBM_STORE_F64_FX) {
        std::snprintf(g_create_err, sizeof(g_create_err),
                      "storage must be LBM_STORE_F64 or LBM_STORE_F64_FX");
        return LBM_ERR_UNSUPPORTED;
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->n = n_cases;
    b->mode = storage == LBM_STORE_F64_FX ? 3 : 0;
    b->stream = (cudaStream_t)stream;
    b->cfg.assign(cfgs, cfgs + n_cases);
    b->hc.resize(n_cases);
    std::vector<DevParticle> recs(n_cases);
    for (int c = 0; c < n_cases; ++c) {
        lbm_status st = make_case(b, c, cfgs[c], particles[c], storage, b->hc[c], recs[c]);
        if (st != LBM_OK) {
            // nothing has been allocated; the message stays readable through
            // lbm_batch_last_error(NULL) on this thread
            std::snprintf(g_create_err, sizeof(g_create_err), "%s", b->err);
            delete b;
            return st;
        }
    }
    b->max_sub = 0;
    b->any_mem = 0;
    b->cell_updates = 0;
    for (auto& c : b->hc) {
        b->max_sub = std::max(b->max_sub, c.subcycles);
        b->any_mem |= c.kind == 2;
        b->cell_updates += c.g.n * c.subcycles;
    }

    // work lists (bulk lists get their items in apply_layout)
    std::vector<int> all(n_cases), mem;
    std::vector<long long> map_it(n_cases), refill_it;
    for (int c = 0; c < n_cases; ++c) {
        all[c] = c;
        map_it[c] = map_items(b->hc[c]);
        if (b->hc[c].kind == 2) {
            mem.push_back(c);
            refill_it.push_back(refill_items(b->hc[c]));
        }
    }
    fill_list(b->map_l, all, map_it);
    fill_list(b->refill_l, mem, refill_it);
    b->near_l.resize(b->max_sub);
    b->bulk_l.resize(b->max_sub);
    for (int s = 0; s < b->max_sub; ++s) {
        std::vector<int> cs;
        std::vector<long long> it, zero;
        for (int c = 0; c < n_cases; ++c)
            if (b->hc[c].subcycles > s) {
                cs.push_back(c);
                it.push_back(b->hc[c].nblk);
                zero.push_back(0);
            }
        fill_list(b->near_l[s], cs, it);
        fill_list(b->bulk_l[s], cs, zero);
    }

    // arena layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    const size_t o_cases = take(sizeof(BatchCase) * n_cases);
    const size_t o_status = take(sizeof(int));
    const size_t o_parts = take(sizeof(DevParticle) * n_cases);
    const size_t o_prev = take(sizeof(DevParticle) * n_cases);
    const size_t o_force = take(sizeof(double) * 6 * n_cases);
    auto list_off = [&](WorkList& w, size_t& ol, size_t& ob) {
        ol = take(sizeof(int) * std::max(w.n, 1));
        ob = take(sizeof(long long) * (w.n + 1));
    };
    size_t ml, mb, rl, rb, ol, ob;
    b->one.n = 1;
    list_off(b->one, ol, ob);
    list_off(b->map_l, ml, mb);
    list_off(b->refill_l, rl, rb);
    std::vector<size_t> nl(b->max_sub), nb(b->max_sub), bl(b->max_sub), bb(b->max_sub);
    for (int s = 0; s < b->max_sub; ++s) {
        list_off(b->near_l[s], nl[s], nb[s]);
        list_off(b->bulk_l[s], bl[s], bb[s]);
    }
    std::vector<size_t> o_buf0(n_cases), o_buf1(n_cases), o_part(n_cases), o_map(n_cases),
        o_chg(n_cases), o_cpart(n_cases);
    for (int c = 0; c < n_cases; ++c) {
        const BatchCase& k = b->hc[c];
        const size_t pdf = sizeof(double) * (size_t)NQ * (size_t)k.g.n;
        o_buf0[c] = take(pdf);
        o_buf1[c] = take(pdf);
        o_part[c] = take(sizeof(double) * 6 * (size_t)k.subcycles * (size_t)k.nblk);
        o_map[c] = take(sizeof(unsigned short) * (size_t)k.map_ext[0] * k.map_ext[1] * k.map_ext[2]);
        o_chg[c] = take(sizeof(double) * 6);
        o_cpart[c] = take(sizeof(double) * 6 * (size_t)refill_blocks(k.refill_side));
    }
    b->arena_bytes = off;

    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    int lo_prio = 0, hi_prio = 0;  // near-sweep branch first in line (see lbm_api.cu)
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, hi_prio);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t1);
    if (e == cudaSuccess) e = cudaMalloc(&b->arena, b->arena_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->arena, 0, b->arena_bytes, b->stream);
    if (e != cudaSuccess) {
        lbm_status st = cuda_fail(b, e, "batch allocation");
        std::snprintf(g_create_err, sizeof(g_create_err), "%s", b->err);
        release(b);
        return st;
    }
    char* base = (char*)b->arena;
    b->dcases = (BatchCase*)(base + o_cases);
    b->dstatus = (int*)(base + o_status);
    b->dparts = (DevParticle*)(base + o_parts);
    b->dprev = (DevParticle*)(base + o_prev);
    b->dforce = (double*)(base + o_force);
    auto bind = [&](WorkList& w, size_t ol, size_t ob) {
        w.list = (int*)(base + ol);
        w.base = (long long*)(base + ob);
    };
    bind(b->one, ol, ob);
    bind(b->map_l, ml, mb);
    bind(b->refill_l, rl, rb);
    for (int s = 0; s < b->max_sub; ++s) {
        bind(b->near_l[s], nl[s], nb[s]);
        bind(b->bulk_l[s], bl[s], bb[s]);
    }
    for (int c = 0; c < n_cases; ++c) {
        BatchCase& k = b->hc[c];
        k.buf[0] = (double*)(base + o_buf0[c]);
        k.buf[1] = (double*)(base + o_buf1[c]);
        k.partials = (double*)(base + o_part[c]);
        k.map = (unsigned short*)(base + o_map[c]);
        k.charge = (double*)(base + o_chg[c]);
        k.charge_part = (double*)(base + o_cpart[c]);
        k.remap_charge = 0;
        k.part = b->dparts + c;
        k.prev = b->dprev + c;
        k.force = b->dforce + 6 * c;
    }
    lbm_status st = LBM_OK;
    e = cudaMemcpyAsync(b->dcases, b->hc.data(), sizeof(BatchCase) * n_cases, cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->dparts, recs.data(), sizeof(DevParticle) * n_cases,
                            cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) st = cuda_fail(b, e, "case upload");
    if (st == LBM_OK) st = upload_list(b, b->map_l);
    if (st == LBM_OK) st = upload_list(b, b->refill_l);
    for (int s = 0; s < b->max_sub && st == LBM_OK; ++s) st = upload_list(b, b->near_l[s]);
    long long max_cells = 0;
    for (auto& k : b->hc) max_cells = std::max(max_cells, k.g.n);
    if (st == LBM_OK && (e = launch_batch_init(b->dcases, n_cases, max_cells, b->stream)) != cudaSuccess)
        st = cuda_fail(b, e, "init launch");
    if (st == LBM_OK) st = apply_layouts(b, std::vector<int>(n_cases, LBM_BATCH_PLANE));
    if (st == LBM_OK) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        b->resident = std::max(sms, 1) * batch_bulk_blocks_per_sm(b->mode);
        b->grid = 0;
        st = build_graph(b);
    }
    if (st != LBM_OK) {
        std::snprintf(g_create_err, sizeof(g_create_err), "%s", b->err);
        release(b);
        return st;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int nsteps) {
    if (!b || nsteps < 0) return LBM_ERR_ARG;
    for (int i = 0; i < nsteps; ++i) BK(b, cudaGraphLaunch(b->exec, b->stream), "graph launch");
    return LBM_OK;
}

lbm_status lbm_batch_set_tuning(lbm_batch* b, const int* layouts, int grid) {
    if (!b) return LBM_ERR_ARG;
    if (grid < 0 || grid > (1 << 24)) return fail(b, LBM_ERR_ARG, "grid must be 0..2^24");
    std::vector<int> lays(b->n, LBM_BATCH_PLANE);
    for (int i = 0; layouts && i < b->n; ++i) {
        if (layouts[i] < LBM_BATCH_BOX32 || layouts[i] > LBM_BATCH_PLANE)
            return fail(b, LBM_ERR_ARG, "layouts must be LBM_BATCH_BOX32..LBM_BATCH_PLANE");
        lays[i] = layouts[i];
    }
    BK(b, cudaStreamSynchronize(b->stream), "tuning sync");
    lbm_status st = apply_layouts(b, lays);
    if (st != LBM_OK) return st;
    b->grid = grid;
    return build_graph(b);
}

lbm_status lbm_batch_autotune(lbm_batch* b, int reps, int* layouts, int* grid, double* ms) {
    if (!b || reps < 1 || reps > 100) return fail(b, LBM_ERR_ARG, "reps must be 1..100");
    BK(b, cudaStreamSynchronize(b->stream), "tuning sync");
    // 1. per case: the layout whose bulk sweep of that case alone is fastest
    std::vector<double> best_t(b->n, 1e300);
    std::vector<int> best_l(b->n, LBM_BATCH_PLANE);
    for (int lay = LBM_BATCH_BOX32; lay <= LBM_BATCH_PLANE; ++lay) {
        lbm_status st = apply_layouts(b, std::vector<int>(b->n, lay));
        if (st != LBM_OK) return st;
        for (int c = 0; c < b->n; ++c) {
            fill_list(b->one, std::vector<int>{c}, std::vector<long long>{bulk_items(b->hc[c].g, lay)});
            if ((st = upload_list(b, b->one)) != LBM_OK) return st;
            double t = 0.0;
            if ((st = time_bulk(b, b->one, 0, reps, &t)) != LBM_OK) return st;  // synchronises
            if (t < best_t[c]) {
                best_t[c] = t;
                best_l[c] = lay;
            }
        }
    }
    lbm_status st = apply_layouts(b, best_l);
    if (st != LBM_OK) return st;
    // 2. for the whole first sweep: one block per tile or a persistent grid
    const int grids[4] = {0, b->resident, 2 * b->resident, 4 * b->resident};
    double best = 1e300;
    int best_g = 0;
    for (int gi = 0; gi < 4; ++gi) {
        double t = 0.0;
        if ((st = time_bulk(b, b->bulk_l[0], grids[gi], reps, &t)) != LBM_OK) return st;
        if (t < best) {
            best = t;
            best_g = grids[gi];
        }
    }
    b->grid = best_g;
    if ((st = build_graph(b)) != LBM_OK) return st;
    if (layouts)
        for (int c = 0; c < b->n; ++c) layouts[c] = best_l[c];
    if (grid) *grid = best_g;
    if (ms) *ms = best;
    return LBM_OK;
}

lbm_status lbm_batch_get_particles(lbm_batch* b, lbm_particle* host_out) {
    if (!b || !host_out) return fail(b, LBM_ERR_ARG, "null output");
    std::vector<DevParticle> recs((size_t)b->n);
    BK(b, cudaMemcpyAsync(recs.data(), b->dparts, sizeof(DevParticle) * b->n,
                          cudaMemcpyDeviceToHost, b->stream),
       "particle download");
    lbm_status st = read_status(b);
    for (int i = 0; i < b->n; ++i) {
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

lbm_status lbm_batch_get_forces(lbm_batch* b, double* F, double* T) {
    if (!b || !F || !T) return fail(b, LBM_ERR_ARG, "null output");
    std::vector<double> ft((size_t)6 * b->n);
    BK(b, cudaMemcpyAsync(ft.data(), b->dforce, sizeof(double) * 6 * b->n, cudaMemcpyDeviceToHost,
                          b->stream),
       "force download");
    lbm_status st = read_status(b);
    for (int i = 0; i < b->n; ++i)
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] = ft[6 * i + a];
            T[3 * i + a] = ft[6 * i + 3 + a];
        }
    return st;
}

lbm_status lbm_batch_get_pdf(lbm_batch* b, int c, double* host_out, size_t bytes) {
    if (!b || !host_out || c < 0 || c >= b->n) return fail(b, LBM_ERR_ARG, "bad case index or output");
    const size_t need = sizeof(double) * (size_t)NQ * (size_t)b->hc[c].g.n;
    if (bytes != need) return fail(b, LBM_ERR_ARG, "byte count does not match the case's PDF field");
    int cur = 0;
    BK(b, cudaMemcpyAsync(&cur, &b->dcases[c].cur, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
       "state index copy");
    BK(b, cudaStreamSynchronize(b->stream), "stream synchronize");
    BK(b, cudaMemcpyAsync(host_out, b->hc[c].buf[cur & 1], need, cudaMemcpyDeviceToHost, b->stream),
       "pdf download");
    return read_status(b);
}

long long lbm_batch_cell_updates(const lbm_batch* b) { return b ? b->cell_updates : 0; }

size_t lbm_batch_device_bytes(const lbm_batch* b) { return b ? b->arena_bytes : 0; }

int lbm_batch_graph_kernels(const lbm_batch* b) { return b ? b->graph_kernels : 0; }

lbm_status lbm_batch_set_remap_charge(lbm_batch* b, int enable) {
    if (!b || (enable != 0 && enable != 1)) return LBM_ERR_ARG;
    BK(b, cudaStreamSynchronize(b->stream), "charge sync");
    int any = 0;
    for (int i = 0; i < b->n; ++i) {
        BatchCase& c = b->hc[i];
        c.remap_charge = c.kind == 2 ? enable : 0;
        any |= c.remap_charge;
        // cur lives on the device and is flipped there: write only this field
        BK(b, cudaMemcpyAsync(&b->dcases[i].remap_charge, &c.remap_charge, sizeof(int),
                              cudaMemcpyHostToDevice, b->stream),
           "case upload");
        BK(b, cudaMemsetAsync(c.charge, 0, sizeof(double) * 6, b->stream), "charge reset");
    }
    BK(b, cudaStreamSynchronize(b->stream), "charge sync");  // host records above
    b->any_charge = any;
    return build_graph(b);
}

lbm_status lbm_batch_profile_enable(lbm_batch* b, int enable) {
    if (!b || (enable != 0 && enable != 1)) return LBM_ERR_ARG;
    if (enable && !b->dprof)
        BK(b, cudaMalloc(&b->dprof, 3 * sizeof(unsigned long long)), "cudaMalloc profile");
    if (b->dprof)
        BK(b, cudaMemsetAsync(b->dprof, 0, 3 * sizeof(unsigned long long), b->stream),
           "profile reset");
    if (enable == b->profiling) return LBM_OK;
    b->profiling = enable;
    return build_graph(b);
}

lbm_status lbm_batch_profile_read(lbm_batch* b, double* bulk_ms, long long* launches) {
    if (!b || !bulk_ms || !launches) return LBM_ERR_ARG;
    unsigned long long h[3] = {0, 0, 0};
    if (b->dprof) {
        BK(b, cudaMemcpyAsync(h, b->dprof, sizeof(h), cudaMemcpyDeviceToHost, b->stream),
           "profile copy");
        BK(b, cudaStreamSynchronize(b->stream), "profile sync");
    }
    *bulk_ms = (double)h[1] * 1e-6;
    *launches = (long long)h[2];
    return read_status(b);
}

lbm_status lbm_batch_synchronize(lbm_batch* b) {
    if (!b) return LBM_ERR_ARG;
    return read_status(b);
}

void lbm_batch_destroy(lbm_batch* b) { release(b); }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : g_create_err; }

}  // extern "C"
