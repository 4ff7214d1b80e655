// Kernels of the coupled D3Q19 step and their launchers (sm_103a).
//
// One global step (Algorithm 1 / Algorithm 2 of Rettinger & Ruede,
// arXiv:1702.04910) is built from:
//   k_bulk      fused pull stream + fluid collision for every cell that no
//               particle comes near (the whole domain but an O(D^3) box);
//   k_near      the same for the cells near a particle, with the coupling:
//               PSM solid fractions and weighted collision Eq. (20)-(26) and
//               force/torque Eq. (28)-(29), or MEM link boundary conditions
//               Eq. (12)/(14) and link forces Eq. (16); per-block force
//               partials reduced warp -> block in a fixed order;
//   k_finalize  fixed-order sum of the block partials, subcycle average;
//   k_rigid     explicit Euler rigid-body update;
//   k_refill    MEM re-mapping: PDF reconstruction Eq. (19) of uncovered
//               cells, then their collision; optionally the momentum the
//               covered and uncovered cells exchange with the fluid, as
//               fixed-order block partials (k_charge_total adds them, and
//               the next k_finalize takes them off the force);
//   k_bulk_pair the 16-bit bulk sweep, two x-neighbours per thread in packed
//               f32x2 arithmetic.
// The batched ensemble has k_batch_* counterparts of these; k_stamp reads
// the global timer around a launch for device-side timing.
#include <cuda_runtime.h>

#include <type_traits>

#include "lbm_launch.h"

namespace lbmgpu {

// ---------------------------------------------------------------------------
// per-cell force/torque slots (a cell may touch up to CELL_SLOTS particles)
struct Slots {
    int id[CELL_SLOTS];
    double v[CELL_SLOTS][6];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int s = 0; s < CELL_SLOTS; ++s) {
            id[s] = -1;
#pragma unroll
            for (int c = 0; c < 6; ++c) v[s][c] = 0.0;
        }
    }
    // returns false when every slot is taken by other particles
    __device__ __forceinline__ bool add(int p, const double (&F)[3], const double (&T)[3]) {
#pragma unroll
        for (int s = 0; s < CELL_SLOTS; ++s) {
            if (id[s] == p || id[s] < 0) {
                id[s] = p;
                v[s][0] += F[0];
                v[s][1] += F[1];
                v[s][2] += F[2];
                v[s][3] += T[0];
                v[s][4] += T[1];
                v[s][5] += T[2];
                return true;
            }
        }
        return false;
    }
    __device__ __forceinline__ double get(int p, int c) const {
        double r = 0.0;
#pragma unroll
        for (int s = 0; s < CELL_SLOTS; ++s)
            if (id[s] == p) r += v[s][c];
        return r;
    }
};

__device__ __forceinline__ void cross3(const double (&a)[3], const double (&b)[3],
                                       double (&r)[3]) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

// ---------------------------------------------------------------------------
// MEM pull for a fluid cell: stream Eq. (2); links whose upstream cell is
// solid take the boundary value Eq. (12) (BB), Eq. (14) (CLI) or Eq. (15)
// (MR, coefficients derived for the TRT link recurrence: kappa_1 = 1,
// kappa_0 = (1 - 2d - 2d^2)/(1+d)^2, kappa_-1 = d^2/(1+d)^2, kappabar_-1 =
// -kappa_0, kappabar_-2 = -kappa_-1, alpha = 4/(1+d)^2, d = delta_q; MR
// falls back to CLI where x - 2 c_q is not fluid, CLI to BB); resting
// closed walls take halfway bounce-back.  When `slots` is non-null the link
// force Eq. (16) and its torque about X_p (arm x_b - X_p) are accumulated.
//
// In pull form the link of the paper (fluid x, solid neighbour x + c_qp)
// appears while filling direction q = qbar_p: the upstream cell x - c_q is
// x + c_qp.
// Owner of a cell: from the per-step map when given, else evaluated from the
// particle records (same predicate, R6).
__device__ __forceinline__ int owner_of(const Geom& g, const DevParticle* parts, int np,
                                        const GeoMap* gm, int x, int y, int z) {
    return gm ? mapped_owner(g, parts, np, *gm, x, y, z) : cell_owner(g, parts, np, x, y, z);
}

// Post-collision momentum j~(x) of the boundary cell, loaded on the first MR
// link of the cell (Eq. (15) correction term).
struct MrCell {
    double j[3];
    bool have;
};

template <typename T>
__device__ __forceinline__ void own_momentum(const T* __restrict__ src, const Geom& g,
                                             long long idx, MrCell& mc) {
    if (mc.have) return;
    double j0 = 0.0, j1 = 0.0, j2 = 0.0;
#pragma unroll
    for (int q = 1; q < NQ; ++q) {
        const double v = ld_pdf(src + (long long)q * g.n + idx, q);
        j0 += v * cx(q);
        j1 += v * cy(q);
        j2 += v * cz(q);
    }
    mc.j[0] = j0;
    mc.j[1] = j1;
    mc.j[2] = j2;
    mc.have = true;
}

// Lattice velocities for a direction known only at run time (the link loop):
// two bits per direction holding c + 1.
template <int A>
__host__ __device__ constexpr unsigned long long c_bits() {
    unsigned long long b = 0;
    for (int q = 0; q < NQ; ++q)
        b |= (unsigned long long)((A == 0 ? cx(q) : (A == 1 ? cy(q) : cz(q))) + 1) << (2 * q);
    return b;
}
__device__ __forceinline__ int rcx(int q) { return (int)((c_bits<0>() >> (2 * q)) & 3ull) - 1; }
__device__ __forceinline__ int rcy(int q) { return (int)((c_bits<1>() >> (2 * q)) & 3ull) - 1; }
__device__ __forceinline__ int rcz(int q) { return (int)((c_bits<2>() >> (2 * q)) & 3ull) - 1; }

// Coordinates of x + sign * c_q (sign = +1 or -1), q known at run time.
__device__ __forceinline__ void shifted_rt(const Nbr& b, int x, int y, int z, int q, int sign,
                                           int& xs, int& ys, int& zs) {
    const int dx = sign * rcx(q), dy = sign * rcy(q), dz = sign * rcz(q);
    xs = dx > 0 ? b.xp : (dx < 0 ? b.xm : x);
    ys = dy > 0 ? b.yp : (dy < 0 ? b.ym : y);
    zs = dz > 0 ? b.zp : (dz < 0 ? b.zm : z);
}

// Phase 1 of the MEM pull, one direction Q: resting wall -> halfway
// bounce-back; fluid upstream cell -> stream Eq. (2); solid upstream cell ->
// bit Q of `cut`, filled by the link loop.
template <typename T, typename C, int Q>
__device__ __forceinline__ void mem_pull_one(const T* __restrict__ src, const Geom& g,
                                             const DevParticle* parts, int np, const GeoMap* gm,
                                             const Nbr& b, int x, int y, int z, long long idx,
                                             C (&f)[NQ], unsigned& cut, int* status) {
    constexpr int QP = opp(Q);
    int xs, ys, zs;
    shifted<Q>(b, x, y, z, -1, xs, ys, zs);
    if (cz(Q) != 0 && (zs < 0 || zs >= g.nz)) {
        f[Q] = PdfStore<T>::template load<C>(src + (long long)QP * g.n + idx, QP);
        return;
    }
    const int owner = owner_of(g, parts, np, gm, xs, ys, zs);
    // index checks: a failure is reported (ST_BOUNDS) and the access skipped
    if (!owner) {
        if (xs < 0 || xs >= g.nx || ys < 0 || ys >= g.ny || zs < 0 || zs >= g.nz) {
            atomicOr(status, ST_BOUNDS);
            f[Q] = (C)0.0;
            return;
        }
        f[Q] = PdfStore<T>::template load<C>(src + (long long)Q * g.n + lin(g, xs, ys, zs), Q);
        return;
    }
    if (owner < 0 || owner > np) {
        atomicOr(status, ST_BOUNDS);
        f[Q] = (C)0.0;
        return;
    }
    cut |= 1u << Q;
}

template <typename T, typename C, int Q>
struct MemPull {
    __device__ __forceinline__ static void run(const T* __restrict__ src, const Geom& g,
                                               const DevParticle* parts, int np, const GeoMap* gm,
                                               const Nbr& b, int x, int y, int z, long long idx,
                                               C (&f)[NQ], unsigned& cut, int* status) {
        mem_pull_one<T, C, Q>(src, g, parts, np, gm, b, x, y, z, idx, f, cut, status);
        MemPull<T, C, Q + 1>::run(src, g, parts, np, gm, b, x, y, z, idx, f, cut, status);
    }
};
template <typename T, typename C>
struct MemPull<T, C, NQ> {
    __device__ __forceinline__ static void run(const T* __restrict__, const Geom&,
                                               const DevParticle*, int, const GeoMap*, const Nbr&,
                                               int, int, int, long long, C (&)[NQ], unsigned&,
                                               int*) {}
};

// Phase 2: the boundary value f_q(x, t+1) of one cut link (q filled at x,
// qp = qbar the paper's link direction towards the solid cell x + c_qp):
// Eq. (12) BB, Eq. (14) CLI or Eq. (15) MR, and, when `ft` is non-null, the
// link force Eq. (16) and its torque about X_p (arm x_b - X_p) in ft[0..5],
// with the owning particle's 1-based index in *owner_out (0: no force).
template <typename T>
__device__ __forceinline__ double mem_link(const T* __restrict__ src, const Geom& g, const Coupl& cp,
                                        const DevParticle* parts, int np, const GeoMap* gm,
                                        const Nbr& b, int x, int y, int z, long long idx, int q,
                                        double* ft, int* owner_out, int* status, MrCell& mc) {
    if (ft) *owner_out = 0;
    const int qp = opp(q);
    const double cqx = rcx(qp), cqy = rcy(qp), cqz = rcz(qp);  // c_qp
    int xs, ys, zs;
    shifted_rt(b, x, y, z, q, -1, xs, ys, zs);  // x - c_q = x + c_qp, solid
    const int owner = owner_of(g, parts, np, gm, xs, ys, zs);
    if (owner < 1 || owner > np) {
        atomicOr(status, ST_BOUNDS);
        return 0.0;
    }
    const DevParticle& P = parts[owner - 1];
    const double xc = x + 0.5, yc = y + 0.5, zc = z + 0.5;
    const double delta =
        cp.variant == 0 ? 0.5 : link_delta(g, P, xc, yc, zc, rcx(qp), rcy(qp), rcz(qp));
    const double xb[3] = {xc + delta * cqx, yc + delta * cqy, zc + delta * cqz};
    double v[3];
    body_velocity(g, P, xb[0], xb[1], xb[2], v[0], v[1], v[2]);
    const double vc = v[0] * cqx + v[1] * cqy + v[2] * cqz;
    const double ftqp = ld_pdf(src + (long long)qp * g.n + idx, qp);  // f~_qp(x)
    const double wr = 3.0 * wq(qp) * cp.rho0;                 // w_q / c_s^2 * rho0
    double val;
    bool cli_done = false;
    if (cp.variant >= 1) {
        // second node x - c_qp = x + c_q must be a fluid cell (CLI and MR)
        int x2, y2, z2;
        shifted_rt(b, x, y, z, q, +1, x2, y2, z2);
        bool ok = !(rcz(q) != 0 && (z2 < 0 || z2 >= g.nz));
        if (ok) ok = owner_of(g, parts, np, gm, x2, y2, z2) == 0;
        if (ok && (x2 < 0 || x2 >= g.nx || y2 < 0 || y2 >= g.ny || z2 < 0 || z2 >= g.nz)) {
            atomicOr(status, ST_BOUNDS);
            ok = false;
        }
        if (ok) {
            const double f2 = ld_pdf(src + (long long)qp * g.n + lin(g, x2, y2, z2), qp);
            const double fq = ld_pdf(src + (long long)q * g.n + idx, q);
            bool mr_done = false;
            if (cp.variant == 2) {
                // Eq. (15): third node x - 2 c_qp = x + 2 c_q must be fluid too
                int x3 = x2 + rcx(q), y3 = y2 + rcy(q), z3 = z2 + rcz(q);
                x3 = x3 < 0 ? x3 + g.nx : (x3 >= g.nx ? x3 - g.nx : x3);
                y3 = y3 < 0 ? y3 + g.ny : (y3 >= g.ny ? y3 - g.ny : y3);
                bool ok3 = true;
                if (g.bc_z) ok3 = z3 >= 0 && z3 < g.nz;
                else z3 = z3 < 0 ? z3 + g.nz : (z3 >= g.nz ? z3 - g.nz : z3);
                if (ok3) ok3 = owner_of(g, parts, np, gm, x3, y3, z3) == 0;
                if (ok3 && (x3 < 0 || x3 >= g.nx || y3 < 0 || y3 >= g.ny || z3 < 0 || z3 >= g.nz)) {
                    atomicOr(status, ST_BOUNDS);
                    ok3 = false;
                }
                if (ok3) {
                    const double f3 = ld_pdf(src + (long long)qp * g.n + lin(g, x3, y3, z3), qp);
                    const double fq2 = ld_pdf(src + (long long)q * g.n + lin(g, x2, y2, z2), q);
                    own_momentum(src, g, idx, mc);
                    const double d1 = (1.0 + delta) * (1.0 + delta);
                    const double k0 = (1.0 - 2.0 * delta - 2.0 * delta * delta) / d1;
                    const double km1 = delta * delta / d1;
                    const double alpha = 4.0 / d1;
                    // (1 - |lambda_-|) n^-_qp(x, t), rebuilt from the stored values
                    const double odd = 0.5 * (ftqp - fq) -
                                       3.0 * wq(qp) * (cqx * mc.j[0] + cqy * mc.j[1] + cqz * mc.j[2]);
                    val = ftqp + k0 * (f2 - fq) + km1 * (f3 - fq2) - alpha * wr * vc +
                          cp.mr_cpc / d1 * odd;
                    mr_done = true;
                }
            }
            if (!mr_done) {
                const double k0 = (1.0 - 2.0 * delta) / (1.0 + 2.0 * delta);
                const double alpha = 4.0 / (1.0 + 2.0 * delta);
                val = ftqp + k0 * f2 - k0 * fq - alpha * wr * vc;
            }
            cli_done = true;
        }
    }
    if (!cli_done) val = ftqp - 2.0 * wr * vc;
    if (ft) {
        double F[3], arm[3], Tq[3];
        F[0] = (cqx - v[0]) * ftqp - (-cqx - v[0]) * val;
        F[1] = (cqy - v[1]) * ftqp - (-cqy - v[1]) * val;
        F[2] = (cqz - v[2]) * ftqp - (-cqz - v[2]) * val;
        separation(g, xb[0], xb[1], xb[2], P, arm[0], arm[1], arm[2]);
        cross3(arm, F, Tq);
        ft[0] = F[0];
        ft[1] = F[1];
        ft[2] = F[2];
        ft[3] = Tq[0];
        ft[4] = Tq[1];
        ft[5] = Tq[2];
        *owner_out = owner;
    }
    return val;
}

template <typename C, int Q>
struct MemMerge {
    __device__ __forceinline__ static void run(unsigned cut, const double (&lv)[NQ], C (&f)[NQ]) {
        if ((cut >> Q) & 1u) f[Q] = (C)lv[Q];
        MemMerge<C, Q + 1>::run(cut, lv, f);
    }
};
template <typename C>
struct MemMerge<C, NQ> {
    __device__ __forceinline__ static void run(unsigned, const double (&)[NQ], C (&)[NQ]) {}
};

// MEM pull for a fluid cell: stream Eq. (2) on every link whose upstream cell
// is fluid (phase 1, unrolled), then the boundary values of the cut links in a
// loop over them (phase 2, one copy of the link code, links in increasing q).
template <typename T, typename C>
__device__ __forceinline__ void mem_pull(const T* __restrict__ src, const Geom& g, const Coupl& cp,
                                         const DevParticle* parts, int np, const GeoMap* gm,
                                         int x, int y, int z, long long idx, C (&f)[NQ],
                                         Slots* slots, int* status) {
    Nbr b = make_nbr(g, x, y, z);
    f[0] = PdfStore<T>::template load<C>(src + idx, 0);
    unsigned cut = 0;
    MemPull<T, C, 1>::run(src, g, parts, np, gm, b, x, y, z, idx, f, cut, status);
    if (cut) {
        double lv[NQ];
        MrCell mc;
        mc.have = false;
        for (unsigned m = cut; m; m &= m - 1) {
            const int q = __ffs(m) - 1;
            double ft[6];
            int owner = 0;
            lv[q] = mem_link(src, g, cp, parts, np, gm, b, x, y, z, idx, q, slots ? ft : nullptr,
                             &owner, status, mc);
            if (slots && owner) {
                const double F[3] = {ft[0], ft[1], ft[2]}, Tq[3] = {ft[3], ft[4], ft[5]};
                if (!slots->add(owner - 1, F, Tq)) atomicOr(status, ST_TOO_MANY_OBJECTS);
            }
        }
        MemMerge<C, 1>::run(cut, lv, f);
    }
}

// Per-warp scratch of the warp-cooperative MEM link loop.
struct LinkWarp {
    double lv[NQ * 32];            // link values, in list order
    double ft[32][6];              // force and torque of the links of one round
    double jt[32][3];              // MR: post-collision momentum of each lane's cell
    long long idx[32];
    int x[32], y[32], z[32], own[32];
    unsigned short list[NQ * 32];  // (lane << 5) | q, lanes in order, q ascending
};

template <typename C, int Q>
struct WarpMerge {
    __device__ __forceinline__ static void run(unsigned cut, const double* lv, int k, C (&f)[NQ]) {
        if ((cut >> Q) & 1u) f[Q] = (C)lv[k++];
        WarpMerge<C, Q + 1>::run(cut, lv, k, f);
    }
};
template <typename C>
struct WarpMerge<C, NQ> {
    __device__ __forceinline__ static void run(unsigned, const double*, int, C (&)[NQ]) {}
};

// Warp-cooperative phase 2 for the near sweep (all 32 lanes call it): the cut
// links of the warp's cells are listed in lane order and spread over the lanes
// 32 at a time, so a boundary cell with many links no longer holds up its
// warp.  Each cell then adds the forces of its own links in ascending q (the
// order of the per-cell loop) and takes its link values.
template <typename T, typename C>
__device__ __forceinline__ void mem_links_warp(const T* __restrict__ src, const Geom& g,
                                               const Coupl& cp, const DevParticle* parts,
                                               const GeoMap* gm, int x, int y, int z, long long idx,
                                               unsigned cut, C (&f)[NQ], Slots& slots, int* status,
                                               LinkWarp& w, int lane) {
    const unsigned full = 0xffffffffu;
    const int nl = __popc(cut);
    int inc = nl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(full, inc, o);
        if (lane >= o) inc += t;
    }
    const int total = __shfl_sync(full, inc, 31);
    if (total == 0) return;  // warp-uniform
    const int first = inc - nl;
    int k = first;
    for (unsigned m = cut; m; m &= m - 1) w.list[k++] = (unsigned short)((lane << 5) | (__ffs(m) - 1));
    w.x[lane] = x;
    w.y[lane] = y;
    w.z[lane] = z;
    w.idx[lane] = idx;
    if (cut && cp.variant == 2) {
        MrCell mc;
        mc.have = false;
        own_momentum(src, g, idx, mc);
        w.jt[lane][0] = mc.j[0];
        w.jt[lane][1] = mc.j[1];
        w.jt[lane][2] = mc.j[2];
    }
    __syncwarp();
    for (int base = 0; base < total; base += 32) {
        const int e = base + lane;
        w.own[lane] = 0;
        if (e < total) {
            const int ol = w.list[e] >> 5, q = w.list[e] & 31;
            const int lx = w.x[ol], ly = w.y[ol], lz = w.z[ol];
            const Nbr b = make_nbr(g, lx, ly, lz);
            MrCell mc;
            mc.have = cp.variant == 2;
            if (mc.have) {
                mc.j[0] = w.jt[ol][0];
                mc.j[1] = w.jt[ol][1];
                mc.j[2] = w.jt[ol][2];
            }
            w.lv[e] = mem_link(src, g, cp, parts, cp.np, gm, b, lx, ly, lz, w.idx[ol], q,
                               &w.ft[lane][0], &w.own[lane], status, mc);
        }
        __syncwarp();
        // this round's links of this lane's cell: entries [lo, hi)
        const int lo = first > base ? first : base;
        const int hi = (first + nl) < (base + 32) ? (first + nl) : (base + 32);
        for (int e2 = lo; e2 < hi; ++e2) {
            const int s = e2 - base;
            if (w.own[s]) {
                const double F[3] = {w.ft[s][0], w.ft[s][1], w.ft[s][2]};
                const double Tq[3] = {w.ft[s][3], w.ft[s][4], w.ft[s][5]};
                if (!slots.add(w.own[s] - 1, F, Tq)) atomicOr(status, ST_TOO_MANY_OBJECTS);
            }
        }
        __syncwarp();
    }
    WarpMerge<C, 1>::run(cut, w.lv, first, f);
    __syncwarp();
}

// ---------------------------------------------------------------------------
// PSM weighted collision Eq. (26) with C^PSM Eq. (20), B1/B2 Eq. (21)/(22),
// M1/M2/M3 Eq. (23)-(25), force/torque Eq. (28)-(29).  `eps[k]` are the
// solid fractions of particles `pid[k]` (k < nobj) at this cell.  Returns
// true when the cell's fluid density is not finite and positive.
template <typename C>
__device__ inline bool psm_collide(C (&f)[NQ], const Coll<C>& k, const Coupl& cp, const Geom& g,
                                   const DevParticle* parts, int nobj, const int (&pid)[CELL_SLOTS],
                                   const double (&eps)[CELL_SLOTS], int x, int y, int z,
                                   Slots& slots) {
    C Cf[NQ], Fq[NQ], ssum[NQ], feqU[NQ];
    C rho, ux, uy, uz;
    fluid_operator(f, k, Cf, Fq, rho, ux, uy, uz);
    equilibrium(rho, ux, uy, uz, k.rho0, feqU);
#pragma unroll
    for (int q = 0; q < NQ; ++q) ssum[q] = (C)0;
    double B = 0.0;
    const double xc = x + 0.5, yc = y + 0.5, zc = z + 0.5;
    for (int o = 0; o < nobj; ++o) {
        const DevParticle& P = parts[pid[o]];
        const double e = eps[o];
        const double Bs =
            cp.variant == 0 ? e : e * (cp.tau - 0.5) / ((1.0 - e) + (cp.tau - 0.5));
        B += Bs;
        double v[3];
        body_velocity(g, P, xc, yc, zc, v[0], v[1], v[2]);
        C feqV[NQ];
        equilibrium(rho, (C)v[0], (C)v[1], (C)v[2], k.rho0, feqV);
        double Fs[3] = {0.0, 0.0, 0.0};
        const C Bc = (C)Bs;
        const C om = (C)(1.0 - 1.0 / cp.tau);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int qb = opp(q);
            C cs;
            if (cp.variant == 0)
                cs = (f[qb] - feqU[qb]) - (f[q] - feqV[q]);
            else if (cp.variant == 1)
                cs = (feqV[q] - f[q]) + om * (f[q] - feqU[q]);
            else
                cs = (f[qb] - feqV[qb]) - (f[q] - feqV[q]);
            ssum[q] += Bc * cs;
            Fs[0] += (double)cs * cx(qb);
            Fs[1] += (double)cs * cy(qb);
            Fs[2] += (double)cs * cz(qb);
        }
        double F[3] = {Bs * Fs[0], Bs * Fs[1], Bs * Fs[2]}, arm[3], Tq[3];
        separation(g, xc, yc, zc, P, arm[0], arm[1], arm[2]);
        cross3(arm, F, Tq);
        slots.add(pid[o], F, Tq);
    }
    const C oneB = (C)(1.0 - B);
#pragma unroll
    for (int q = 0; q < NQ; ++q) f[q] = f[q] + (oneB * Cf[q] + ssum[q]) + oneB * Fq[q];
    return density_bad(rho);
}

// ---------------------------------------------------------------------------
// bulk sweep: every cell outside the near-particle regions.  Tiles that no
// region touches skip the per-cell test (block-uniform branch).
// Resident 256-thread blocks per SM requested for k_bulk (at most 85
// registers per thread).
template <typename C> struct BulkBlocks { static constexpr int value = 3; };

// One tile (tX, tY, tZ) of the bulk sweep for the calling thread (tx, ty).
template <typename T, typename C, bool NOSTREAM, int CPT>
__device__ __forceinline__ void bulk_tile(const T* __restrict__ src, T* __restrict__ dst,
                                          const Geom& g, const Coll<C>& k,
                                          const DevParticle* __restrict__ parts, int np,
                                          int all_tiles, int tX, int tY, int tZ, int tx, int ty,
                                          int* __restrict__ status) {
    bool near_tile = false;
    if (!all_tiles) {
        for (int s = 0; s < np && !near_tile; ++s)
            near_tile = tile_in_reg(g, parts[s].reg, tX, tY, tZ);
    }
    const int x = tX * g.tx + tx, y = tY * g.ty + ty;
    if (x >= g.nx || y >= g.ny) return;
    // CPT cells per thread along z: all their loads are issued before the
    // first collision, doubling the bytes in flight of the 32-bit sweep
    C f[CPT][NQ];
    bool act[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int z = tZ * CPT + c;
        act[c] = z < g.nz;
        if (act[c] && near_tile)
            for (int s = 0; s < np; ++s)
                if (cell_in_reg(g, parts[s].reg, x, y, z)) act[c] = false;  // k_near's cell
        if (act[c]) {
            const long long idx = lin(g, x, y, z);
            if (NOSTREAM)
                load_own(src, g, idx, f[c]);
            else
                pull_plain(src, g, x, y, z, idx, f[c]);
        }
    }
    bool bad = false;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        if (!act[c]) continue;
        const int z = tZ * CPT + c;
        bad |= collide_fluid(f[c], k);
        store_own(dst, g, lin(g, x, y, z), f[c]);
    }
    if (bad) atomicOr(status, ST_FLUID);
}

template <typename T, typename C, bool NOSTREAM, int CPT>
__global__ void __launch_bounds__(256, BulkBlocks<C>::value)
    k_bulk(const T* __restrict__ src, T* __restrict__ dst, Geom g, Coll<C> k,
           const DevParticle* __restrict__ parts, int np, int all_tiles, int* __restrict__ status) {
    bulk_tile<T, C, NOSTREAM, CPT>(src, dst, g, k, parts, np, all_tiles, blockIdx.x, blockIdx.y,
                                   blockIdx.z, threadIdx.x, threadIdx.y, status);
}

// ---------------------------------------------------------------------------
// 16-bit shifted storage, two x-neighbours per thread.  The pair (x0, x0 + 1),
// x0 even, is read and written as one 32-bit word per direction (nx even, so
// every row starts on a 4-byte boundary); a pull across x takes the two
// aligned words around the shifted pair and selects its halves with a byte
// permute.  Conversions use the packed two-value forms.  The collision runs on
// the stored shifted values g_q = f_q - w_q themselves: with rho = 1 + sum_q
// g_q and j = sum_q g_q c_q (sum_q w_q c_q = 0), the folded update
// f' = alpha f + beta fbar - (P +- M) becomes g' = alpha g + beta gbar -
// (P +- M) with rho replaced by sum_q g_q in P (alpha + beta - 1 = lambda_+
// cancels the l+ w_q term), so the same collide_fluid code applies with no
// shift on load or store, and FP32 rounds the small deviations, not f.
template <typename T> struct Pair16;
template <>
struct Pair16<__half> {
    __device__ __forceinline__ static float2 unpack(unsigned u) {
        __half2 h;
        memcpy(&h, &u, 4);
        return __half22float2(h);
    }
    __device__ __forceinline__ static unsigned pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        unsigned u;
        memcpy(&u, &h, 4);
        return u;
    }
    __device__ __forceinline__ static __half one(float a) { return __float2half_rn(a); }
};
template <>
struct Pair16<__nv_bfloat16> {
    __device__ __forceinline__ static float2 unpack(unsigned u) {
        __nv_bfloat162 h;
        memcpy(&h, &u, 4);
        return __bfloat1622float2(h);
    }
    __device__ __forceinline__ static unsigned pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        unsigned u;
        memcpy(&u, &h, 4);
        return u;
    }
    __device__ __forceinline__ static __nv_bfloat16 one(float a) { return __float2bfloat16_rn(a); }
};

__device__ __forceinline__ unsigned ld_word(const void* p) {
    return __ldg(reinterpret_cast<const unsigned*>(p));
}

// direction Q of the pair at row `row` (= lin(0, y, z)); xm2 / xp2 are the
// (periodic) even columns left / right of x0
template <typename T, int Q>
__device__ __forceinline__ void pull_pair_one(const T* __restrict__ src, const Geom& g,
                                              const NbrOff& o, long long row, int x0, int xm2,
                                              int xp2, f2 (&f)[NQ]) {
    float2 v;
    if ((cz(Q) > 0 && o.zlo) || (cz(Q) < 0 && o.zhi)) {
        v = Pair16<T>::unpack(ld_word(src + (long long)opp(Q) * g.n + row + x0));  // halfway BB
    } else {
        long long r = row;
        if (cy(Q) > 0) r += o.dym;
        else if (cy(Q) < 0) r += o.dyp;
        if (cz(Q) > 0) r += o.dzm;
        else if (cz(Q) < 0) r += o.dzp;
        const T* a = src + (long long)Q * g.n + r;
        if (cx(Q) == 0) {
            v = Pair16<T>::unpack(ld_word(a + x0));
        } else if (cx(Q) > 0) {  // cells x0 - 1, x0
            v = Pair16<T>::unpack(__byte_perm(ld_word(a + xm2), ld_word(a + x0), 0x5432));
        } else {  // cells x0 + 1, x0 + 2
            v = Pair16<T>::unpack(__byte_perm(ld_word(a + x0), ld_word(a + xp2), 0x5432));
        }
    }
    f[Q] = f2(v);  // shifted values g_q (see above), cell x0 in lane x
}

template <typename T, int Q>
struct PullPair {
    __device__ __forceinline__ static void run(const T* __restrict__ src, const Geom& g,
                                               const NbrOff& o, long long row, int x0, int xm2,
                                               int xp2, f2 (&f)[NQ]) {
        pull_pair_one<T, Q>(src, g, o, row, x0, xm2, xp2, f);
        PullPair<T, Q + 1>::run(src, g, o, row, x0, xm2, xp2, f);
    }
};
template <typename T>
struct PullPair<T, NQ> {
    __device__ __forceinline__ static void run(const T* __restrict__, const Geom&, const NbrOff&,
                                               long long, int, int, int, f2 (&)[NQ]) {}
};

// Grid (ceil(nx / (2 PAIR_TX)), ceil(ny / PAIR_TY), nz), block (PAIR_TX, PAIR_TY).
// One row of 128 cells per 64-thread block: the near-particle sweep runs
// beside this kernel and each of its blocks holds 7.7k (MEM) to 11.5k (PSM)
// registers; with small bulk blocks an SM that hosts near blocks gives up
// only as many bulk warps as their registers need (measured in the 128 x 128
// x 512 step, FP16: 0.70 of HBM with 64 x 4, 0.745 with 64 x 2, 0.76 with
// 64 x 1; 32 x 1 and 128 x 1 are slower).
constexpr int PAIR_TX = 64, PAIR_TY = 1;

template <typename T>
__global__ void __launch_bounds__(PAIR_TX * PAIR_TY, 768 / (PAIR_TX * PAIR_TY))
    k_bulk_pair(const T* __restrict__ src, T* __restrict__ dst, Geom g, Coll<float> k,
                const DevParticle* __restrict__ parts, int np, int* __restrict__ status) {
    const int bx0 = 2 * blockIdx.x * PAIR_TX, by0 = blockIdx.y * PAIR_TY;
    const int x0 = bx0 + 2 * threadIdx.x;
    const int y = by0 + threadIdx.y, z = blockIdx.z;
    if (x0 >= g.nx || y >= g.ny) return;
    // k_near's cells are left alone; a block whose cells no region reaches
    // (block-uniform test) skips the per-cell one
    bool near_a = false, near_b = false;
    for (int s = 0; s < np; ++s) {
        const int* r = parts[s].reg;
        if (!in_range(z, r[8], r[9], g.nz) ||
            !spans_meet(by0, min(PAIR_TY, g.ny - by0), r[4], r[5], g.ny) ||
            !spans_meet(bx0, min(2 * PAIR_TX, g.nx - bx0), r[0], r[1], g.nx))
            continue;
        near_a = near_a || cell_in_reg(g, r, x0, y, z);
        near_b = near_b || cell_in_reg(g, r, x0 + 1, y, z);
    }
    if (near_a && near_b) return;
    const NbrOff o = make_off(g, x0, y, z);
    const long long row = lin(g, 0, y, z);
    const int xm2 = x0 == 0 ? g.nx - 2 : x0 - 2;
    const int xp2 = x0 + 2 == g.nx ? 0 : x0 + 2;
    // both cells collide in the two lanes of the packed f32x2 arithmetic
    f2 f[NQ];
    PullPair<T, 0>::run(src, g, o, row, x0, xm2, xp2, f);
    const unsigned bad = collide_fluid<f2, true>(f, k);
    if (((bad & 1u) && !near_a) || ((bad & 2u) && !near_b)) atomicOr(status, ST_FLUID);
    if (!near_a && !near_b) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            *reinterpret_cast<unsigned*>(dst + (long long)q * g.n + row + x0) =
                Pair16<T>::pack(f[q].v.x, f[q].v.y);
    } else {
        const long long idx = row + x0 + (near_a ? 1 : 0);
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            dst[(long long)q * g.n + idx] = Pair16<T>::one(near_a ? f[q].v.y : f[q].v.x);
    }
}

// ---------------------------------------------------------------------------
// near-particle sweep over the cell region of each particle (cells within
// R + NEAR_HALO of the centre per axis).  Grid (bx, by, bz * np) of
// NEAR_BX x NEAR_BY x NEAR_BZ blocks: block (bx, by, bz) of particle p covers
// region offsets [bx*NEAR_BX, ...) etc.; a cell that also lies in the region
// of a lower-index particle is left to that particle's blocks.  Each block
// writes, for every particle q, its fixed-order force/torque sum to
// partials[((p * nblk + blk) * np + q) * 6 + c].
// One near-kernel block: region offsets (bx, by, bzz) of particle p, whose
// force/torque sums land in partials[((p * nblk + blk) * np + q) * 6 + c].
// `sp` holds the particle records in shared memory; every thread of the
// block must call this (it synchronises for the reduction).
// MEM: a cell whose centre lies farther than R + 3/2 from every sphere centre
// has no solid neighbour (neighbour centres are at most sqrt(2) away and a
// cell is solid iff its centre is within R, R6), so its pull is the plain one.
__device__ __forceinline__ bool clear_of_particles(const Geom& g, const DevParticle* sp, int np,
                                                   int x, int y, int z) {
    const double xc = x + 0.5, yc = y + 0.5, zc = z + 0.5;
    for (int s = 0; s < np; ++s) {
        double dx, dy, dz;
        separation(g, xc, yc, zc, sp[s], dx, dy, dz);
        const double r = sp[s].r + 1.5;
        if (dx * dx + dy * dy + dz * dz <= r * r) return false;
    }
    return true;
}

template <typename T, typename C, int KIND, bool NOSTREAM>
__device__ __forceinline__ void near_block(const T* __restrict__ src, T* __restrict__ dst,
                                           const Geom& g, const Coll<C>& k, const Coupl& cp,
                                           const DevParticle* sp, const GeoMap& gm,
                                           double* __restrict__ partials, int* __restrict__ status,
                                           int p, int bx, int by, int bzz, long long nblk,
                                           long long blk, double (*red)[6], LinkWarp* lw) {
    const int tid = threadIdx.x + NEAR_BX * (threadIdx.y + NEAR_BY * threadIdx.z);
    constexpr int nthr = NEAR_BX * NEAR_BY * NEAR_BZ;
    const int* R = sp[p].reg;
    const int kx = bx * NEAR_BX + threadIdx.x, ky = by * NEAR_BY + threadIdx.y,
              kz = bzz * NEAR_BZ + threadIdx.z;
    bool active = kx < R[1] && ky < R[5] && kz < R[9];
    int x = R[0] + kx, y = R[4] + ky, z = R[8] + kz;
    if (x >= g.nx) x -= g.nx;
    if (y >= g.ny) y -= g.ny;
    if (z >= g.nz) z -= g.nz;
    if (active)
        for (int s = 0; s < p; ++s)
            if (cell_in_reg(g, sp[s].reg, x, y, z)) active = false;
    Slots slots;
    slots.clear();
    if (active && (x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz)) {
        atomicOr(status, ST_BOUNDS);
        active = false;
    }
    if (active) {
        const long long idx = lin(g, x, y, z);
        C f[NQ];
        if (KIND == 2) {
            // MEM with no stream (first sweep after set-up): fluid cells collide
            if (NOSTREAM && !map_at(gm, p, kx, ky, kz)) {
                load_own(src, g, idx, f);
                if (collide_fluid(f, k)) atomicOr(status, ST_FLUID);
                store_own(dst, g, idx, f);
            }
        } else {
            if (NOSTREAM)
                load_own(src, g, idx, f);
            else
                pull_plain(src, g, x, y, z, idx, f);
            int nobj = 0;
            int pid[CELL_SLOTS];
            double eps[CELL_SLOTS];
            if (KIND == 1) {
                const double n3 = (double)cp.subsample * cp.subsample * cp.subsample;
                for (int s = 0; s < cp.np; ++s) {
                    int ox, oy, oz;
                    if (!region_offsets(g, sp[s].reg, x, y, z, ox, oy, oz)) continue;
                    const int cnt = map_at(gm, s, ox, oy, oz);
                    if (cnt == 0) continue;
                    const double e = (double)cnt / n3;
                    if (nobj < CELL_SLOTS) {
                        pid[nobj] = s;
                        eps[nobj] = e;
                        ++nobj;
                    } else {
                        atomicOr(status, ST_TOO_MANY_OBJECTS);
                    }
                }
            }
            const bool bad = nobj == 0
                                 ? collide_fluid(f, k)
                                 : psm_collide(f, k, cp, g, sp, nobj, pid, eps, x, y, z, slots);
            if (bad) atomicOr(status, ST_FLUID);
            store_own(dst, g, idx, f);
        }
    }
    if (KIND == 2 && !NOSTREAM) {
        // MEM (Sec. 2.2): solid cells are not updated; every lane of the warp
        // takes part in the link loop, cells or not
        C f[NQ];
        bool fluid = false;
        long long idx = 0;
        unsigned cut = 0;
        if (active && !map_at(gm, p, kx, ky, kz)) {
            fluid = true;
            idx = lin(g, x, y, z);
            if (clear_of_particles(g, sp, cp.np, x, y, z)) {
                pull_plain(src, g, x, y, z, idx, f);  // no solid neighbour, no link
            } else {
                const Nbr b = make_nbr(g, x, y, z);
                f[0] = PdfStore<T>::template load<C>(src + idx, 0);
                MemPull<T, C, 1>::run(src, g, sp, cp.np, &gm, b, x, y, z, idx, f, cut, status);
            }
        }
        mem_links_warp(src, g, cp, sp, &gm, x, y, z, idx, cut, f, slots, status, lw[tid >> 5],
                       tid & 31);
        if (fluid) {
            if (collide_fluid(f, k)) atomicOr(status, ST_FLUID);
            store_own(dst, g, idx, f);
        }
    }
    if (KIND == 0 || (NOSTREAM && KIND == 2)) return;
    // fixed-order reduction of this block's contribution for each particle
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr / 32;
    for (int q = 0; q < cp.np; ++q) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double v = warp_sum(slots.get(q, c));
            if (lane == 0) red[warp][c] = v;
        }
        __syncthreads();
        if (tid < 6) {
            double acc = 0.0;
            for (int w = 0; w < nwarp; ++w) acc += red[w][tid];
            if (p < cp.np && blk < nblk) partials[(((long long)p * nblk + blk) * cp.np + q) * 6 + tid] = acc;
            else atomicOr(status, ST_BOUNDS);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// near-particle sweep over the cell region of each particle (cells within
// R + NEAR_HALO of the centre per axis).  Grid (bx, by, bz * np) of
// NEAR_BX x NEAR_BY x NEAR_BZ blocks: block (bx, by, bz) of particle p covers
// region offsets [bx*NEAR_BX, ...) etc.; a cell that also lies in the region
// of a lower-index particle is left to that particle's blocks.
template <typename T, typename C, int KIND, bool NOSTREAM>
__global__ void __launch_bounds__(256)
    k_near(const T* __restrict__ src, T* __restrict__ dst, Geom g, Coll<C> k, Coupl cp,
           const DevParticle* __restrict__ parts, GeoMap gm, double* __restrict__ partials,
           int* __restrict__ status, int bz) {
    __shared__ DevParticle sp[MAX_PARTICLES];
    __shared__ double red[8][6];
    __shared__ LinkWarp lw[KIND == 2 ? NEAR_BX * NEAR_BY * NEAR_BZ / 32 : 1];
    const int tid = threadIdx.x + NEAR_BX * (threadIdx.y + NEAR_BY * threadIdx.z);
    constexpr int nthr = NEAR_BX * NEAR_BY * NEAR_BZ;
    for (int i = tid; i < cp.np * (int)(sizeof(DevParticle) / sizeof(double)); i += nthr)
        reinterpret_cast<double*>(sp)[i] = reinterpret_cast<const double*>(parts)[i];
    __syncthreads();
    const int p = blockIdx.z / bz, bzz = blockIdx.z % bz;
    const long long nblk = (long long)gridDim.x * gridDim.y * bz;
    const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * bzz);
    near_block<T, C, KIND, NOSTREAM>(src, dst, g, k, cp, sp, gm, partials, status, p, blockIdx.x,
                                     blockIdx.y, bzz, nblk, blk, red, lw);
}

// ---------------------------------------------------------------------------
// Per-step geometry map (computed once per global step, before the sweeps):
// for every cell of particle p's region, MEM: the owner under the current
// particle state (0 fluid, s+1 inside particle s, lowest s first, R6);
// PSM: the number of the n^3 supersamples inside particle p (R15).  The
// sweeps then read these instead of re-evaluating FP64 geometry per link.
// Grid (ceil(ex/32), ey, ez * np), 32 threads per block.
// Called by all 32 lanes of a warp that covers 32 consecutive kx of one row
// (ky, kz the same on every lane).  PSM: cells wholly outside or inside the
// sphere take the quick count; the warp then samples each remaining cell of
// the row together (two of the 64 samples per lane for n = 4), so a row costs
// a few cooperative sample sets instead of one 64-sample loop per lane.
template <int KIND>
__device__ __forceinline__ void map_cell(const Geom& g, const Coupl& cp, const DevParticle* sp,
                                         unsigned short* __restrict__ map, int ex, int ey, int ez,
                                         int p, int kx, int ky, int kz) {
    const int* R = sp[p].reg;
    const bool valid = kx < R[1] && ky < R[5] && kz < R[9];
    int x = R[0] + kx, y = R[4] + ky, z = R[8] + kz;
    if (x >= g.nx) x -= g.nx;
    if (y >= g.ny) y -= g.ny;
    if (z >= g.nz) z -= g.nz;
    unsigned short* out = map + (((long long)p * ez + kz) * ey + ky) * ex + kx;
    if (KIND == 2) {
        if (valid) *out = (unsigned short)cell_owner(g, sp, cp.np, x, y, z);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int quick = valid ? solid_count_quick(g, sp[p], x, y, z, cp.subsample) : 0;
    if (valid && quick >= 0) *out = (unsigned short)quick;
    unsigned todo = __ballot_sync(0xffffffffu, valid && quick < 0);
    while (todo) {
        const int c = __ffs(todo) - 1;
        todo &= todo - 1;
        const int xc = __shfl_sync(0xffffffffu, x, c);
        const int cnt = solid_count_warp(g, sp[p], xc, y, z, cp.subsample, lane);
        if (lane == c) *out = (unsigned short)cnt;
    }
}

template <int KIND>
__global__ void __launch_bounds__(32)
    k_map(Geom g, Coupl cp, const DevParticle* __restrict__ parts, unsigned short* __restrict__ map,
          int ex, int ey, int ez) {
    __shared__ DevParticle sp[MAX_PARTICLES];
    const int nd = cp.np * (int)(sizeof(DevParticle) / sizeof(double));
    for (int i = threadIdx.x; i < nd; i += blockDim.x)
        reinterpret_cast<double*>(sp)[i] = reinterpret_cast<const double*>(parts)[i];
    __syncthreads();
    map_cell<KIND>(g, cp, sp, map, ex, ey, ez, blockIdx.z / ez, blockIdx.x * 32 + threadIdx.x,
                   blockIdx.y, blockIdx.z % ez);
}

// ---------------------------------------------------------------------------
// fixed-order force/torque total of particle q (one block per particle):
// F = (S_1 + ... + S_nsub) / nsub with S_k the sum, over the near-kernel
// blocks of every particle's region, of subcycle k's partials for q.
// charge != nullptr: the pending re-mapping momentum charge of q, [q][6],
// divided by the step's lattice time nsub, is taken off.
__device__ __forceinline__ void finalize_block(int np, long long nblk,
                                               const double* __restrict__ partials, int nsub,
                                               double* __restrict__ out, int q,
                                               double (*red)[6],
                                               const double* __restrict__ charge = nullptr) {
    const int tid = threadIdx.x;
    const long long count = (long long)np * nblk;
    double tot[6] = {0, 0, 0, 0, 0, 0};
    for (int sub = 0; sub < nsub; ++sub) {
        const double* base = partials + (long long)sub * count * np * 6;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (long long kk = tid; kk < count; kk += blockDim.x) {
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[c] += base[(kk * np + q) * 6 + c];
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) red[tid][c] = acc[c];
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (tid < s)
#pragma unroll
                for (int c = 0; c < 6; ++c) red[tid][c] += red[tid + s][c];
            __syncthreads();
        }
        if (tid == 0)
#pragma unroll
            for (int c = 0; c < 6; ++c) tot[c] += red[0][c];
        __syncthreads();
    }
    if (tid == 0)
        for (int c = 0; c < 6; ++c)
            out[q * 6 + c] = charge ? tot[c] / nsub - charge[q * 6 + c] / nsub : tot[c] / nsub;
}

__global__ void __launch_bounds__(256)
    k_finalize(int np, long long nblk, const double* __restrict__ partials, int nsub,
               double* __restrict__ out, const double* __restrict__ charge) {
    __shared__ double red[256][6];
    finalize_block(np, nblk, partials, nsub, out, blockIdx.x, red, charge);
}

// ---------------------------------------------------------------------------
// explicit Euler rigid-body update over dt, gravity + buoyancy
// (rho_p - rho0) V g; keeps the previous state in `prev`.
__device__ __forceinline__ void rigid_one(const Geom& g, DevParticle* __restrict__ part,
                                          DevParticle* __restrict__ prev,
                                          const double* __restrict__ force, double rho0, double gx,
                                          double gy, double gz, double dt, int wall_contact,
                                          int* __restrict__ status) {
    DevParticle P = *part;
    *prev = P;
    if (P.fixed == 0.0) {
        const double PI = 3.14159265358979323846;
        const double D = P.d, R = 0.5 * D;
        const double V = PI * D * D * D / 6.0;
        const double m = P.rho * V, I = m * D * D / 10.0;
        const double grav[3] = {gx, gy, gz};
        double Ft[3];
        for (int a = 0; a < 3; ++a) Ft[a] = force[a] + (P.rho - rho0) * V * grav[a];
        for (int a = 0; a < 3; ++a) P.x[a] += dt * P.u[a];
        for (int a = 0; a < 3; ++a) P.u[a] += dt * Ft[a] / m;
        for (int a = 0; a < 3; ++a) P.w[a] += dt * force[3 + a] / I;
        // a non-finite state, or a surface moving a cell or more per step,
        // is outside what the lattice can represent: report it and keep the
        // previous state so that the cell geometry stays well defined
        bool sane = true;
        for (int a = 0; a < 3; ++a)
            sane = sane && isfinite(P.x[a]) && fabs(P.u[a]) < 1.0 && fabs(P.w[a]) * R < 1.0;
        if (!sane) {
            atomicOr(status, ST_UNSTABLE);
            P = *prev;
        }
        const double L[3] = {(double)g.nx, (double)g.ny, (double)g.nz};
        for (int a = 0; a < 3; ++a) {
            if (a == 2 && g.bc_z) continue;
            if (P.x[a] < 0.0) P.x[a] += L[a];
            else if (P.x[a] >= L[a]) P.x[a] -= L[a];
        }
        if (g.bc_z == 2) {
            // open boundaries: the near region must stay clear of them
            if (P.x[2] - R - OPEN_MARGIN < 0.0 || P.x[2] + R + OPEN_MARGIN > L[2])
                atomicOr(status, ST_DOMAIN);
        } else if (g.bc_z) {
            if (wall_contact) {
                if (P.x[2] - R < 1.0) {
                    P.x[2] = R + 1.0;
                    if (P.u[2] < 0.0) P.u[2] = 0.0;
                }
                if (P.x[2] + R > L[2] - 1.0) {
                    P.x[2] = L[2] - 1.0 - R;
                    if (P.u[2] > 0.0) P.u[2] = 0.0;
                }
            } else if (P.x[2] - R < 0.0 || P.x[2] + R > L[2]) {
                atomicOr(status, ST_DOMAIN);
            }
        }
    }
    store_region(g, P);
    *part = P;
}

// explicit Euler rigid-body update over dt, gravity + buoyancy
// (rho_p - rho0) V g; keeps the previous state in `prev`.
__global__ void k_rigid(Geom g, DevParticle* __restrict__ parts, DevParticle* __restrict__ prev,
                        int np, const double* __restrict__ force, double rho0, double gx,
                        double gy, double gz, double dt, int wall_contact,
                        int* __restrict__ status) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    rigid_one(g, parts + p, prev + p, force + 6 * p, rho0, gx, gy, gz, dt, wall_contact, status);
}

__global__ void k_regions(Geom g, DevParticle* parts, int np) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) store_region(g, parts[p]);
}

// ---------------------------------------------------------------------------
// MEM re-mapping with PDF reconstruction (Sec. 2.2, Eq. (19)).  One thread per
// cell of the box around each particle's old position finds the candidates: a
// cell solid under p_old (owner p) and fluid under p_new.  Each candidate is
// then rebuilt by its whole warp (refill_warp) and gets:
//   extrapolate = 1: f = 3 f(x+c_n) - 3 f(x+2c_n) + f(x+3c_n) (fewer terms when
//     fewer usable fluid cells follow), with the pre-collision values of those
//     cells rebuilt from srcB (the buffer the last sweep pulled from) under
//     p_old; then the velocity constraint j = rho0 v; with no usable cell,
//     f_eq(rho_bar, v);
//   extrapolate = 0: f_eq(rho0, v);
// and is then collided (plain fluid collision) into dst.

// Pre-collision value f_q(x) of one direction q (known at run time) of a
// fluid cell x, as mem_pull rebuilds it (particle owners from the records).
template <typename T, typename C>
__device__ __forceinline__ C mem_pull_dir(const T* __restrict__ src, const Geom& g, const Coupl& cp,
                                          const DevParticle* parts, int x, int y, int z, int q,
                                          int* status) {
    const long long idx = lin(g, x, y, z);
    if (q == 0) return PdfStore<T>::template load<C>(src + idx, 0);
    const Nbr b = make_nbr(g, x, y, z);
    const int qp = opp(q);
    int xs, ys, zs;
    shifted_rt(b, x, y, z, q, -1, xs, ys, zs);
    if (rcz(q) != 0 && (zs < 0 || zs >= g.nz))
        return PdfStore<T>::template load<C>(src + (long long)qp * g.n + idx, qp);
    const int owner = cell_owner(g, parts, cp.np, xs, ys, zs);
    if (!owner) {
        if (xs < 0 || xs >= g.nx || ys < 0 || ys >= g.ny || zs < 0 || zs >= g.nz) {
            atomicOr(status, ST_BOUNDS);
            return (C)0.0;
        }
        return PdfStore<T>::template load<C>(src + (long long)q * g.n + lin(g, xs, ys, zs), q);
    }
    if (owner < 0 || owner > cp.np) {
        atomicOr(status, ST_BOUNDS);
        return (C)0.0;
    }
    MrCell mc;
    mc.have = false;
    int unused = 0;
    return (C)mem_link(src, g, cp, parts, cp.np, (const GeoMap*)nullptr, b, x, y, z, idx, q,
                       (double*)nullptr, &unused, status, mc);
}

// Per-warp scratch of the refill.
struct RefillWarp {
    double f[3][NQ];  // pre-collision values of the extrapolation cells
    double r[NQ];     // densities of the usable neighbours (no extrapolation cell)
    int ok[NQ];
};

// Rebuilds candidate cell (x, y, z) of particle p; all 32 lanes call it with
// the same cell.  The pulls are spread over the lanes, the rest is computed
// by every lane alike and lane 0 stores.  jm receives the momentum
// sum_q c_q f_q of the rebuilt pre-collision populations (every lane).
template <typename T, typename C>
__device__ __forceinline__ void refill_warp(const T* __restrict__ srcB, T* __restrict__ dst,
                                            const Geom& g, const Coll<C>& k, const Coupl& cp,
                                            const DevParticle* so, const DevParticle* sn,
                                            int extrapolate, int p, int x, int y, int z,
                                            int* __restrict__ status, RefillWarp& w, int lane,
                                            double (&jm)[3]) {
    const DevParticle& Pn = sn[p];
    const double xc = x + 0.5, yc = y + 0.5, zc = z + 0.5;
    double v[3];
    body_velocity(g, Pn, xc, yc, zc, v[0], v[1], v[2]);
    C fn[NQ];
    int m = 0;
    int qn = 1;
    int nbx[3], nby[3], nbz[3];
    if (extrapolate) {
        double nrm[3];
        separation(g, xc, yc, zc, Pn, nrm[0], nrm[1], nrm[2]);
        double len = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        if (len > 0.0)
            for (int a = 0; a < 3; ++a) nrm[a] /= len;
        double best = -1e300;
        for (int q = 1; q < NQ; ++q) {
            double d = nrm[0] * cx(q) + nrm[1] * cy(q) + nrm[2] * cz(q);
            if (d > best) {
                best = d;
                qn = q;
            }
        }
        for (int kk = 1; kk <= 3; ++kk) {
            int xx = wrap_i(x + kk * cx(qn), g.nx), yy = wrap_i(y + kk * cy(qn), g.ny),
                zz = z + kk * cz(qn);
            if (g.bc_z) {
                if (zz < 0 || zz >= g.nz) break;
            } else {
                zz = wrap_i(zz, g.nz);
            }
            if (cell_owner(g, so, cp.np, xx, yy, zz) || cell_owner(g, sn, cp.np, xx, yy, zz))
                break;
            nbx[m] = xx;
            nby[m] = yy;
            nbz[m] = zz;
            ++m;
        }
    }
    if (m > 0) {
        // the m x 19 pulls, lane by lane
        for (int i = lane; i < m * NQ; i += 32) {
            const int jn = i / NQ, q = i - jn * NQ;
            w.f[jn][q] =
                (double)mem_pull_dir<T, C>(srcB, g, cp, so, nbx[jn], nby[jn], nbz[jn], q, status);
        }
        __syncwarp();
        if (m == 1) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) fn[q] = (C)w.f[0][q];
        } else if (m == 2) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) fn[q] = (C)2 * (C)w.f[0][q] - (C)w.f[1][q];
        } else {
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                fn[q] = (C)3 * (C)w.f[0][q] - (C)3 * (C)w.f[1][q] + (C)w.f[2][q];
        }
        // velocity constraint: only the momentum moment changes (sum_q c_qa^2 = 10)
        double j[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            j[0] += (double)fn[q] * cx(q);
            j[1] += (double)fn[q] * cy(q);
            j[2] += (double)fn[q] * cz(q);
        }
        double dj[3];
        for (int a = 0; a < 3; ++a) dj[a] = cp.rho0 * v[a] - j[a];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            fn[q] = (C)((double)fn[q] + (cx(q) * dj[0] + cy(q) * dj[1] + cz(q) * dj[2]) / 10.0);
    } else {
        double rbar = cp.rho0;
        if (extrapolate) {
            // lane q - 1 pulls neighbour x + c_q (q = 1..18) when it is usable
            if (lane < NQ - 1) {
                const int q = lane + 1;
                int xx = wrap_i(x + rcx(q), g.nx), yy = wrap_i(y + rcy(q), g.ny), zz = z + rcz(q);
                bool ok = true;
                if (g.bc_z) ok = zz >= 0 && zz < g.nz;
                else zz = wrap_i(zz, g.nz);
                if (ok)
                    ok = !cell_owner(g, so, cp.np, xx, yy, zz) && !cell_owner(g, sn, cp.np, xx, yy, zz);
                double r = 0.0;
                if (ok) {
                    C fq[NQ];
                    mem_pull(srcB, g, cp, so, cp.np, (const GeoMap*)nullptr, xx, yy, zz,
                             lin(g, xx, yy, zz), fq, (Slots*)nullptr, status);
#pragma unroll
                    for (int qq = 0; qq < NQ; ++qq) r += (double)fq[qq];
                }
                w.r[q] = r;
                w.ok[q] = ok ? 1 : 0;
            }
            __syncwarp();
            double sum = 0.0;
            int cnt = 0;
            for (int q = 1; q < NQ; ++q) {
                if (!w.ok[q]) continue;
                sum += w.r[q];
                ++cnt;
            }
            if (cnt > 0) rbar = sum / cnt;
        }
        equilibrium((C)rbar, (C)v[0], (C)v[1], (C)v[2], k.rho0, fn);
    }
    jm[0] = jm[1] = jm[2] = 0.0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        jm[0] += (double)fn[q] * cx(q);
        jm[1] += (double)fn[q] * cy(q);
        jm[2] += (double)fn[q] * cz(q);
    }
    collide_fluid(fn, k);
    if (lane == 0) {
        if (x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz)
            atomicOr(status, ST_BOUNDS);
        else
            store_own(dst, g, lin(g, x, y, z), fn);
    }
    __syncwarp();
}

// Adds sign * (j, (x_c - X_p) x j) of cell (x, y, z) to acc, X_p the centre
// of P (minimum image in periodic directions).
__device__ __forceinline__ void add_cell_moment(double (&acc)[6], const Geom& g,
                                                const DevParticle& P, int x, int y, int z,
                                                const double (&j)[3], double sign) {
    double r[3];
    separation(g, x + 0.5, y + 0.5, z + 0.5, P, r[0], r[1], r[2]);
    acc[0] += sign * j[0];
    acc[1] += sign * j[1];
    acc[2] += sign * j[2];
    acc[3] += sign * (r[1] * j[2] - r[2] * j[1]);
    acc[4] += sign * (r[2] * j[0] - r[0] * j[2]);
    acc[5] += sign * (r[0] * j[1] - r[1] * j[0]);
}

// Candidate test of thread lid of particle p's box, then the warp's
// candidates one after another.  Every lane of the warp must call this.
// acc != nullptr: re-mapping momentum charge of particle p (uncovered cells
// plus, covered cells minus; moments about the new centre) added to this
// thread's six sums.  The box holds every cell of the new sphere while the
// centre moves by less than 1.5 cells per axis in a step.
template <typename T, typename C>
__device__ __forceinline__ void refill_cells(const T* __restrict__ srcB, T* __restrict__ dst,
                                             const Geom& g, const Coll<C>& k, const Coupl& cp,
                                             const DevParticle* so, const DevParticle* sn,
                                             int extrapolate, int side, int p, long long lid,
                                             int* __restrict__ status, RefillWarp& w, int lane,
                                             double (*acc)[6] = nullptr) {
    bool cand = lid < (long long)side * side * side;
    int x = 0, y = 0, z = 0;
    if (cand) {
        const int kx = (int)(lid % side), ky = (int)((lid / side) % side),
                  kz = (int)(lid / ((long long)side * side));
        const DevParticle& Po = so[p];
        x = (int)floor(Po.x[0] - Po.r) - 1 + kx;
        y = (int)floor(Po.x[1] - Po.r) - 1 + ky;
        z = (int)floor(Po.x[2] - Po.r) - 1 + kz;
        x = wrap_i(x, g.nx);
        y = wrap_i(y, g.ny);
        if (g.bc_z) {
            if (z < 0 || z >= g.nz) cand = false;
        } else {
            z = wrap_i(z, g.nz);
        }
    }
    const int own_old = cand ? cell_owner(g, so, cp.np, x, y, z) : -1;
    const bool test_new = own_old == p + 1 || (acc && own_old == 0);
    const int own_new = test_new ? cell_owner(g, sn, cp.np, x, y, z) : -1;
    cand = own_old == p + 1 && own_new == 0;
    if (acc && own_old == 0 && own_new == p + 1) {
        // covered: the fluid momentum of its pre-collision populations leaves the fluid
        C f[NQ];
        mem_pull(srcB, g, cp, so, cp.np, (const GeoMap*)nullptr, x, y, z, lin(g, x, y, z), f,
                 (Slots*)nullptr, status);
        double j[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            j[0] += (double)f[q] * cx(q);
            j[1] += (double)f[q] * cy(q);
            j[2] += (double)f[q] * cz(q);
        }
        add_cell_moment(*acc, g, sn[p], x, y, z, j, -1.0);
    }
    const unsigned full = 0xffffffffu;
    for (unsigned m = __ballot_sync(full, cand); m; m &= m - 1) {
        const int src_lane = __ffs(m) - 1;
        const int cxl = __shfl_sync(full, x, src_lane), cyl = __shfl_sync(full, y, src_lane),
                  czl = __shfl_sync(full, z, src_lane);
        double jm[3];
        refill_warp<T, C>(srcB, dst, g, k, cp, so, sn, extrapolate, p, cxl, cyl, czl, status, w,
                          lane, jm);
        if (acc && lane == src_lane) add_cell_moment(*acc, g, sn[p], cxl, cyl, czl, jm, 1.0);
    }
}

// The refill box holds the new sphere only for a step of less than 1.5
// cells per axis: a faster step is reported as unstable.
__device__ __forceinline__ void charge_step_check(const Geom& g, const DevParticle& Pn,
                                                  const DevParticle& Po, int* status) {
    double d[3];
    separation(g, Pn.x[0], Pn.x[1], Pn.x[2], Po, d[0], d[1], d[2]);
    if (fabs(d[0]) >= 1.5 || fabs(d[1]) >= 1.5 || fabs(d[2]) >= 1.5) atomicOr(status, ST_UNSTABLE);
}

// Fixed-order sum of the block's per-thread charge sums into out[0..6): a
// butterfly within each warp, then the warps in turn.  Every thread of the
// REFILL_THREADS-thread block calls it.
__device__ __forceinline__ void charge_block_sum(const double (&acc)[6], double* out) {
    __shared__ double red[REFILL_THREADS / 32][6];
    const int tid = threadIdx.x, lane = tid & 31;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        double v = acc[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[tid >> 5][c] = v;
    }
    __syncthreads();
    if (tid < 6) {
        double t = 0.0;
        for (int wi = 0; wi < REFILL_THREADS / 32; ++wi) t += red[wi][tid];
        out[tid] = t;
    }
}

// Grid (ceil(side^3 / REFILL_THREADS), np).  charge_part != nullptr: block
// (bx, p) also writes its fixed-order sums of particle p's re-mapping
// momentum charge to charge_part[(p * gridDim.x + bx) * 6 + c].
template <typename T, typename C>
__global__ void __launch_bounds__(REFILL_THREADS)
    k_refill(const T* __restrict__ srcB, T* __restrict__ dst, Geom g, Coll<C> k, Coupl cp,
             const DevParticle* __restrict__ p_old, const DevParticle* __restrict__ p_new,
             int extrapolate, int side, int* __restrict__ status,
             double* __restrict__ charge_part) {
    __shared__ DevParticle so[MAX_PARTICLES], sn[MAX_PARTICLES];
    const int tid = threadIdx.x;
    const int nd = cp.np * (int)(sizeof(DevParticle) / sizeof(double));
    for (int i = tid; i < nd; i += blockDim.x) {
        reinterpret_cast<double*>(so)[i] = reinterpret_cast<const double*>(p_old)[i];
        reinterpret_cast<double*>(sn)[i] = reinterpret_cast<const double*>(p_new)[i];
    }
    __syncthreads();
    __shared__ RefillWarp rw[REFILL_THREADS / 32];
    const int p = blockIdx.y, lane = tid & 31;
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    refill_cells<T, C>(srcB, dst, g, k, cp, so, sn, extrapolate, side, p,
                       (long long)blockIdx.x * blockDim.x + tid, status, rw[tid >> 5], lane,
                       charge_part ? &acc : nullptr);
    if (!charge_part) return;
    if (tid == 0) charge_step_check(g, sn[p], so[p], status);
    charge_block_sum(acc, charge_part + ((long long)p * gridDim.x + blockIdx.x) * 6);
}

// out[p * 6 + c] = sum over the nblk refill blocks of particle p, in order.
__global__ void k_charge_total(int np, long long nblk, const double* __restrict__ part,
                               double* __restrict__ out) {
    const int t = threadIdx.x;
    if (t >= 6 * np) return;
    const int p = t / 6, c = t - 6 * (t / 6);
    double s = 0.0;
    for (long long b = 0; b < nblk; ++b) s += part[((long long)p * nblk + b) * 6 + c];
    out[t] = s;
}

// ---------------------------------------------------------------------------
// macroscopic fields of the pre-collision state at the start of the next step
// what: 2 rho, 3 u, 4 eps (PSM), 5 owner flag (MEM)
template <typename T, typename C, bool NOSTREAM>
__global__ void __launch_bounds__(256)
    k_macro(const T* __restrict__ state, Geom g, Coll<C> k, Coupl cp,
            const DevParticle* __restrict__ parts, double fx, double fy, double fz, int what,
            void* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((long long)g.nx * g.ny));
    const double xc = x + 0.5, yc = y + 0.5, zc = z + 0.5;
    double* od = reinterpret_cast<double*>(out);
    if (cp.kind == 2) {
        int own = cell_owner(g, parts, cp.np, x, y, z);
        if (what == 5) {
            reinterpret_cast<int*>(out)[i] = own;
            return;
        }
        if (what == 4) {
            od[i] = own ? 1.0 : 0.0;
            return;
        }
        double rho, u[3];
        if (own) {
            rho = cp.rho0;
            body_velocity(g, parts[own - 1], xc, yc, zc, u[0], u[1], u[2]);
        } else {
            // post-collision moments: rho is conserved, j gains f_ext
            double r = 0.0, j[3] = {0.0, 0.0, 0.0};
            for (int q = 0; q < NQ; ++q) {
                double v = ld_pdf(state + (long long)q * g.n + i, q);
                r += v;
                j[0] += v * cx(q);
                j[1] += v * cy(q);
                j[2] += v * cz(q);
            }
            rho = r;
            u[0] = (j[0] - fx) / cp.rho0 + fx / (2.0 * cp.rho0);
            u[1] = (j[1] - fy) / cp.rho0 + fy / (2.0 * cp.rho0);
            u[2] = (j[2] - fz) / cp.rho0 + fz / (2.0 * cp.rho0);
        }
        if (what == 2) od[i] = rho;
        else {
            od[3 * i + 0] = u[0];
            od[3 * i + 1] = u[1];
            od[3 * i + 2] = u[2];
        }
        return;
    }
    if (what == 5) {
        reinterpret_cast<int*>(out)[i] = 0;
        return;
    }
    double B = 0.0, vs[3] = {0.0, 0.0, 0.0}, epsum = 0.0;
    if (cp.kind == 1) {
        for (int s = 0; s < cp.np; ++s) {
            if (!cell_in_reg(g, parts[s].reg, x, y, z)) continue;
            double e = solid_fraction(g, parts[s], x, y, z, cp.subsample);
            if (e <= 0.0) continue;
            epsum += e;
            double Bs = cp.variant == 0 ? e : e * (cp.tau - 0.5) / ((1.0 - e) + (cp.tau - 0.5));
            double v[3];
            body_velocity(g, parts[s], xc, yc, zc, v[0], v[1], v[2]);
            B += Bs;
            for (int a = 0; a < 3; ++a) vs[a] += Bs * v[a];
        }
    }
    if (what == 4) {
        od[i] = epsum;
        return;
    }
    C f[NQ];
    if (NOSTREAM)
        load_own(state, g, i, f);
    else
        pull_plain(state, g, x, y, z, i, f);
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        r += (double)f[q];
        j[0] += (double)f[q] * cx(q);
        j[1] += (double)f[q] * cy(q);
        j[2] += (double)f[q] * cz(q);
    }
    if (what == 2) {
        od[i] = r;
        return;
    }
    const double fe[3] = {fx, fy, fz};
    for (int a = 0; a < 3; ++a) {
        double ua = j[a] / cp.rho0 + fe[a] / (2.0 * cp.rho0);
        od[3 * i + a] = (1.0 - B) * ua + vs[a];
    }
}

template <typename T>
__global__ void k_init_eq(T* __restrict__ dst, Geom g, double rho, double ux, double uy, double uz,
                         double rho0) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    double e[NQ];
    equilibrium(rho, ux, uy, uz, rho0, e);
#pragma unroll
    for (int q = 0; q < NQ; ++q) dst[(long long)q * g.n + i] = PdfStore<T>::template save<double>(e[q], q);
}

template <typename T>
__global__ void k_to_f64(const T* __restrict__ in, double* __restrict__ out, long long count,
                         long long ncell) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = ld_pdf(in + i, (int)(i / ncell));
}

template <typename T>
__global__ void k_from_f64(const double* __restrict__ in, T* __restrict__ out, long long count,
                           long long ncell) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = PdfStore<T>::template save<double>(in[i], (int)(i / ncell));
}


// ---------------------------------------------------------------------------
// Batched ensemble kernels.  Each launch covers every case of a work list;
// block (or work item) t belongs to case list[i] with base[i] <= t < base[i+1].
__device__ __forceinline__ int find_item(const long long* __restrict__ base, int n, long long t) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(base + mid) <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename C>
__device__ __forceinline__ const Coll<C>& batch_coll(const BatchCase& B);
template <>
__device__ __forceinline__ const Coll<double>& batch_coll<double>(const BatchCase& B) {
    return B.kd;
}
template <>
__device__ __forceinline__ const Coll<fx64>& batch_coll<fx64>(const BatchCase& B) {
    return B.kfx;
}

// cell and tile ranges of each case's particle (after upload or a change of
// the bulk tiling); the previous state starts equal to the current one
__global__ void k_batch_regions(BatchCase* __restrict__ cases, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    store_region(cases[c].g, *cases[c].part);
    *cases[c].prev = *cases[c].part;
}

// f = f_eq(rho0, 0) in the stored buffer of every case (fluid at rest: the
// post-collision and pre-collision fields coincide).
__global__ void k_batch_init(BatchCase* __restrict__ cases) {
    const BatchCase& B = cases[blockIdx.y];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.g.n) return;
    double e[NQ];
    equilibrium(B.kd.rho0, 0.0, 0.0, 0.0, B.kd.rho0, e);
#pragma unroll
    for (int q = 0; q < NQ; ++q) B.buf[B.cur][(long long)q * B.g.n + i] = e[q];
}

// geometry map: 32-thread blocks over (x chunk, y, z) of each case's region
__global__ void __launch_bounds__(32) k_batch_map(BatchCase* __restrict__ cases, BatchList l) {
    __shared__ DevParticle sp[1];
    const int i = find_item(l.base, l.n, blockIdx.x);
    const BatchCase& B = cases[l.list[i]];
    const long long local = blockIdx.x - l.base[i];
    for (int k = threadIdx.x; k < (int)(sizeof(DevParticle) / sizeof(double)); k += 32)
        reinterpret_cast<double*>(sp)[k] = reinterpret_cast<const double*>(B.part)[k];
    __syncthreads();
    const int nbx = (B.map_ext[0] + 31) / 32;
    const int bx = (int)(local % nbx);
    const long long rest = local / nbx;
    const int ky = (int)(rest % B.map_ext[1]), kz = (int)(rest / B.map_ext[1]);
    if (B.kind == 2)
        map_cell<2>(B.g, B.cp, sp, B.map, B.map_ext[0], B.map_ext[1], B.map_ext[2], 0,
                    bx * 32 + threadIdx.x, ky, kz);
    else
        map_cell<1>(B.g, B.cp, sp, B.map, B.map_ext[0], B.map_ext[1], B.map_ext[2], 0,
                    bx * 32 + threadIdx.x, ky, kz);
}

// near-particle sweep: one near block of one case per thread block
__global__ void __launch_bounds__(256)
    k_batch_near(BatchCase* __restrict__ cases, BatchList l, int sub, int* __restrict__ status) {
    __shared__ DevParticle sp[1];
    __shared__ double red[8][6];
    __shared__ LinkWarp lw[NEAR_BX * NEAR_BY * NEAR_BZ / 32];
    const int i = find_item(l.base, l.n, blockIdx.x);
    const BatchCase& B = cases[l.list[i]];
    const long long local = blockIdx.x - l.base[i];
    const int tid = threadIdx.x + NEAR_BX * (threadIdx.y + NEAR_BY * threadIdx.z);
    for (int k = tid; k < (int)(sizeof(DevParticle) / sizeof(double)); k += NEAR_BX * NEAR_BY * NEAR_BZ)
        reinterpret_cast<double*>(sp)[k] = reinterpret_cast<const double*>(B.part)[k];
    __syncthreads();
    const int bx = (int)(local % B.box[0]);
    const int by = (int)((local / B.box[0]) % B.box[1]);
    const int bzz = (int)(local / ((long long)B.box[0] * B.box[1]));
    const GeoMap gm{B.map, B.map_ext[0], B.map_ext[1], B.map_ext[2]};
    const int cur = B.cur;
    double* partials = B.partials + (long long)sub * B.nblk * 6;
    if (B.kind == 2)
        near_block<double, double, 2, false>(B.buf[cur], B.buf[1 - cur], B.g, B.kd, B.cp, sp, gm,
                                             partials, status, 0, bx, by, bzz, B.nblk, local, red,
                                             lw);
    else
        near_block<double, double, 1, false>(B.buf[cur], B.buf[1 - cur], B.g, B.kd, B.cp, sp, gm,
                                             partials, status, 0, bx, by, bzz, B.nblk, local, red,
                                             lw);
}

// One 256-cell segment of an xy plane of the bulk sweep: cells
// l = seg * 256 + t (x fastest) of plane z.  Domains whose nx is not a
// multiple of the warp width keep every lane busy (box tiles of tx cells
// leave tx - nx mod tx lanes of each row idle).
template <typename C>
__device__ __forceinline__ void bulk_segment(const double* __restrict__ src,
                                             double* __restrict__ dst, const Geom& g,
                                             const Coll<C>& k, const int* reg, int seg, int z,
                                             int t, int* __restrict__ status) {
    const int l = seg * 256 + t;
    if (l >= g.nx * g.ny) return;
    const int y = l / g.nx, x = l - y * g.nx;
    if (cell_in_reg(g, reg, x, y, z)) return;  // k_batch_near's cell
    const long long idx = lin(g, x, y, z);
    C f[NQ];
    pull_plain(src, g, x, y, z, idx, f);
    if (collide_fluid(f, k)) atomicOr(status, ST_FLUID);
    store_own(dst, g, idx, f);
}

// One tile of case B in its bulk layout (see k_batch_bulk).
template <typename C>
__device__ __forceinline__ void batch_tile(const BatchCase& B, long long local,
                                           int* __restrict__ status) {
    const int cur = B.cur;
    if (B.layout == 1) {
        const int nseg = (B.g.nx * B.g.ny + 255) / 256;
        bulk_segment<C>(B.buf[cur], B.buf[1 - cur], B.g, batch_coll<C>(B), B.part->reg,
                        (int)(local % nseg), (int)(local / nseg), threadIdx.x, status);
    } else {
        const int tX = (int)(local % B.g.ntx);
        const int tY = (int)((local / B.g.ntx) % B.g.nty);
        const int tZ = (int)(local / ((long long)B.g.ntx * B.g.nty));
        bulk_tile<double, C, false, 1>(B.buf[cur], B.buf[1 - cur], B.g, batch_coll<C>(B), B.part, 1,
                                       0, tX, tY, tZ, threadIdx.x % B.g.tx, threadIdx.x / B.g.tx,
                                       status);
    }
}

// bulk sweep: persistent 256-thread blocks striding over the tiles of all
// listed cases.  Each case has its own tiling (B.layout, chosen by the
// autotuner): 0 box tiles of g.tx x g.ty cells (thread t -> (t mod g.tx,
// t / g.tx)); 1 plane segments of 256 cells.  MODE: 0 FP64, 3 fixed-point
// collision.
template <int MODE>
__global__ void __launch_bounds__(256, 3)
    k_batch_bulk(BatchCase* __restrict__ cases, BatchList l, long long total,
                 int* __restrict__ status) {
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = find_item(l.base, l.n, t);
        const BatchCase& B = cases[l.list[i]];
        const long long local = t - l.base[i];
        if (MODE == 3) batch_tile<fx64>(B, local, status);
        else batch_tile<double>(B, local, status);
    }
}

__global__ void k_batch_swap(BatchCase* __restrict__ cases, BatchList l) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < l.n) cases[l.list[i]].cur ^= 1;
}

__global__ void __launch_bounds__(256) k_batch_finalize(BatchCase* __restrict__ cases) {
    __shared__ double red[256][6];
    const BatchCase& B = cases[blockIdx.x];
    const int nsub = B.kind != 0 ? B.subcycles : 1;
    finalize_block(1, B.nblk, B.partials, nsub, B.force, 0, red,
                   B.remap_charge ? B.charge : nullptr);
}

__global__ void k_batch_rigid(BatchCase* __restrict__ cases, int n, int* __restrict__ status) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const BatchCase& B = cases[c];
    const double dt = B.kind != 0 ? (double)B.subcycles : 1.0;
    rigid_one(B.g, B.part, B.prev, B.force, B.kd.rho0, B.gravity[0], B.gravity[1], B.gravity[2],
              dt, B.wall_contact, status);
}

// MEM re-mapping and refilling after the step (reads the buffer the last
// sweep pulled from, writes the stored state)
__global__ void __launch_bounds__(REFILL_THREADS)
    k_batch_refill(BatchCase* __restrict__ cases, BatchList l, int* __restrict__ status) {
    __shared__ DevParticle so[1], sn[1];
    const int i = find_item(l.base, l.n, blockIdx.x);
    const BatchCase& B = cases[l.list[i]];
    const long long local = blockIdx.x - l.base[i];
    for (int k = threadIdx.x; k < (int)(sizeof(DevParticle) / sizeof(double)); k += blockDim.x) {
        reinterpret_cast<double*>(so)[k] = reinterpret_cast<const double*>(B.prev)[k];
        reinterpret_cast<double*>(sn)[k] = reinterpret_cast<const double*>(B.part)[k];
    }
    __syncthreads();
    const int cur = B.cur;
    __shared__ RefillWarp rw[REFILL_THREADS / 32];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    refill_cells<double, double>(B.buf[1 - cur], B.buf[cur], B.g, B.kd, B.cp, so, sn, 1,
                                 B.refill_side, 0, local * blockDim.x + threadIdx.x, status,
                                 rw[threadIdx.x >> 5], threadIdx.x & 31,
                                 B.remap_charge ? &acc : nullptr);
    // re-mapping charge: block partial `local` of this case (see k_refill)
    if (!B.remap_charge) return;
    if (threadIdx.x == 0) charge_step_check(B.g, sn[0], so[0], status);
    charge_block_sum(acc, B.charge_part + local * 6);
}

// Per case with the charge on: charge[c] = the fixed-order total of its
// refill-block partials.  One thread per (case, component).
__global__ void k_batch_charge_total(BatchCase* __restrict__ cases, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 6 * n) return;
    const BatchCase& B = cases[t / 6];
    if (!B.remap_charge) return;
    const int c = t % 6;
    const long long nb = refill_blocks(B.refill_side);
    double s = 0.0;
    for (long long k = 0; k < nb; ++k) s += B.charge_part[k * 6 + c];
    B.charge[c] = s;
}

// ---------------------------------------------------------------------------
// launchers
namespace {
template <typename T, typename C>
const Coll<C>& coll_of(const Launch& L);
template <>
const Coll<double>& coll_of<double, double>(const Launch& L) {
    return L.kd;
}
template <>
const Coll<float>& coll_of<float, float>(const Launch& L) {
    return L.kf;
}
template <>
const Coll<dfloat>& coll_of<double, dfloat>(const Launch& L) {
    return L.kff;
}
template <>
const Coll<fx64>& coll_of<double, fx64>(const Launch& L) {
    return L.kfx;
}

template <typename T, typename C, int CPT>
cudaError_t bulk_cpt(const void* src, void* dst, const Launch& L) {
    dim3 grid(L.g.ntx, L.g.nty, L.g.ntz);
    const auto& k = coll_of<typename std::conditional<(sizeof(T) < 4), C, T>::type, C>(L);
    if (L.nostream)
        k_bulk<T, C, true, CPT><<<grid, L.block, 0, L.stream>>>(
            (const T*)src, (T*)dst, L.g, k, L.parts, L.cp.np, L.all_tiles, L.status);
    else
        k_bulk<T, C, false, CPT><<<grid, L.block, 0, L.stream>>>(
            (const T*)src, (T*)dst, L.g, k, L.parts, L.cp.np, L.all_tiles, L.status);
    return cudaGetLastError();
}

// FP64-state sweeps are arithmetic bound and use one cell per thread; the
// 16/32-bit sweeps are memory bound and take two z cells per thread.
template <typename T, typename C = T>
cudaError_t bulk_t(const void* src, void* dst, const Launch& L) {
    if constexpr (sizeof(T) == 2) {
        // 16-bit sweep with two x-neighbours per thread: even nx, streaming,
        // no open boundaries (those planes take the per-cell kernel)
        if (!L.nostream && L.g.nx % 2 == 0 && L.g.bc_z != 2) {
            dim3 grid((L.g.nx + 2 * PAIR_TX - 1) / (2 * PAIR_TX), (L.g.ny + PAIR_TY - 1) / PAIR_TY,
                      L.g.nz);
            k_bulk_pair<T><<<grid, dim3(PAIR_TX, PAIR_TY, 1), 0, L.stream>>>(
                (const T*)src, (T*)dst, L.g, L.kf, L.parts, L.all_tiles ? 0 : L.cp.np, L.status);
            return cudaGetLastError();
        }
    }
    if constexpr (sizeof(T) <= 4) {
        if (L.g.tz == 2) return bulk_cpt<T, C, 2>(src, dst, L);
    }
    return bulk_cpt<T, C, 1>(src, dst, L);
}

template <typename T, int KIND>
cudaError_t near_kind(const void* src, void* dst, const Launch& L) {
    using C = typename ComputeOf<T>::type;
    dim3 grid(L.box[0], L.box[1], L.box[2] * L.cp.np);
    dim3 block(NEAR_BX, NEAR_BY, NEAR_BZ);
    const auto& k = coll_of<C, C>(L);
    const GeoMap gm{L.map, L.map_ext[0], L.map_ext[1], L.map_ext[2]};
    if (L.nostream)
        k_near<T, C, KIND, true><<<grid, block, 0, L.stream>>>(
            (const T*)src, (T*)dst, L.g, k, L.cp, L.parts, gm, L.partials, L.status, L.box[2]);
    else
        k_near<T, C, KIND, false><<<grid, block, 0, L.stream>>>(
            (const T*)src, (T*)dst, L.g, k, L.cp, L.parts, gm, L.partials, L.status, L.box[2]);
    return cudaGetLastError();
}

template <typename T>
cudaError_t near_t(const void* src, void* dst, const Launch& L) {
    if (L.cp.np <= 0) return cudaSuccess;
    if (L.cp.kind == 1) return near_kind<T, 1>(src, dst, L);
    if (L.cp.kind == 2) return near_kind<T, 2>(src, dst, L);
    return near_kind<T, 0>(src, dst, L);
}

template <typename T>
cudaError_t refill_t(const void* srcB, void* dst, const Launch& L, const DevParticle* po,
                     const DevParticle* pn, int extrapolate, double* charge_part) {
    using C = typename ComputeOf<T>::type;
    if (L.cp.np <= 0) return cudaSuccess;
    int side = L.box[0];  // set by the caller: cube side in cells
    dim3 grid((unsigned)refill_blocks(side), L.cp.np, 1);
    k_refill<T, C><<<grid, REFILL_THREADS, 0, L.stream>>>((const T*)srcB, (T*)dst, L.g, coll_of<C, C>(L),
                                                L.cp, po, pn, extrapolate, side, L.status,
                                                charge_part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t macro_t(const void* state, const Launch& L, int what, void* out) {
    using C = typename ComputeOf<T>::type;
    unsigned blocks = (unsigned)((L.g.n + 255) / 256);
    const auto& k = coll_of<C, C>(L);
    const double fx = L.kd.fx, fy = L.kd.fy, fz = L.kd.fz;
    if (L.nostream)
        k_macro<T, C, true><<<blocks, 256, 0, L.stream>>>((const T*)state, L.g, k, L.cp, L.parts,
                                                          fx, fy, fz, what, out);
    else
        k_macro<T, C, false><<<blocks, 256, 0, L.stream>>>((const T*)state, L.g, k, L.cp, L.parts,
                                                           fx, fy, fz, what, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t init_eq_t(void* dst, const Launch& L, double rho, double ux, double uy, double uz) {
    unsigned blocks = (unsigned)((L.g.n + 255) / 256);
    k_init_eq<T><<<blocks, 256, 0, L.stream>>>((T*)dst, L.g, rho, ux, uy, uz, L.kd.rho0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t to_f64_t(const void* in, double* out, long long count, long long ncell,
                     cudaStream_t s) {
    unsigned blocks = (unsigned)((count + 255) / 256);
    k_to_f64<T><<<blocks, 256, 0, s>>>((const T*)in, out, count, ncell);
    return cudaGetLastError();
}

template <typename T>
cudaError_t from_f64_t(const double* in, void* dst, long long count, long long ncell,
                       cudaStream_t s) {
    unsigned blocks = (unsigned)((count + 255) / 256);
    k_from_f64<T><<<blocks, 256, 0, s>>>(in, (T*)dst, count, ncell);
    return cudaGetLastError();
}
}  // namespace

// storage codes: ST_F64 0, ST_F32 1, ST_F16 4, ST_BF16 5 (FP64 is also the
// state of the float-float (2) and fixed-point (3) bulk modes)
cudaError_t launch_bulk(int storage, const void* src, void* dst, const Launch& L) {
    switch (storage) {
        case 2: return bulk_t<double, dfloat>(src, dst, L);
        case 3: return bulk_t<double, fx64>(src, dst, L);
        case 1: return bulk_t<float>(src, dst, L);
        case 4: return bulk_t<__half, float>(src, dst, L);
        case 5: return bulk_t<__nv_bfloat16, float>(src, dst, L);
        default: return bulk_t<double>(src, dst, L);
    }
}
cudaError_t launch_near(int storage, const void* src, void* dst, const Launch& L) {
    switch (storage) {
        case 1: return near_t<float>(src, dst, L);
        case 4: return near_t<__half>(src, dst, L);
        case 5: return near_t<__nv_bfloat16>(src, dst, L);
        default: return near_t<double>(src, dst, L);
    }
}
cudaError_t launch_refill(int storage, const void* srcB, void* dst, const Launch& L,
                          const DevParticle* p_old, const DevParticle* p_new, int extrapolate,
                          double* charge_part) {
    switch (storage) {
        case 1: return refill_t<float>(srcB, dst, L, p_old, p_new, extrapolate, charge_part);
        case 4: return refill_t<__half>(srcB, dst, L, p_old, p_new, extrapolate, charge_part);
        case 5:
            return refill_t<__nv_bfloat16>(srcB, dst, L, p_old, p_new, extrapolate, charge_part);
        default: return refill_t<double>(srcB, dst, L, p_old, p_new, extrapolate, charge_part);
    }
}
cudaError_t launch_charge_total(const Launch& L, const double* charge_part, double* charge) {
    if (L.cp.np <= 0) return cudaSuccess;
    k_charge_total<<<1, 6 * MAX_PARTICLES, 0, L.stream>>>(L.cp.np, refill_blocks(L.box[0]),
                                                          charge_part, charge);
    return cudaGetLastError();
}
cudaError_t launch_macro(int storage, const void* state, const Launch& L, int what, void* out) {
    switch (storage) {
        case 1: return macro_t<float>(state, L, what, out);
        case 4: return macro_t<__half>(state, L, what, out);
        case 5: return macro_t<__nv_bfloat16>(state, L, what, out);
        default: return macro_t<double>(state, L, what, out);
    }
}
cudaError_t launch_init_eq(int storage, void* dst, const Launch& L, double rho, double ux,
                           double uy, double uz) {
    switch (storage) {
        case 1: return init_eq_t<float>(dst, L, rho, ux, uy, uz);
        case 4: return init_eq_t<__half>(dst, L, rho, ux, uy, uz);
        case 5: return init_eq_t<__nv_bfloat16>(dst, L, rho, ux, uy, uz);
        default: return init_eq_t<double>(dst, L, rho, ux, uy, uz);
    }
}
cudaError_t launch_to_f64(int storage, const void* in, double* out, long long count,
                          long long ncell, cudaStream_t s) {
    switch (storage) {
        case 1: return to_f64_t<float>(in, out, count, ncell, s);
        case 4: return to_f64_t<__half>(in, out, count, ncell, s);
        case 5: return to_f64_t<__nv_bfloat16>(in, out, count, ncell, s);
        default:
            return cudaMemcpyAsync(out, in, sizeof(double) * count, cudaMemcpyDeviceToDevice, s);
    }
}
cudaError_t launch_from_f64(int storage, const double* in, void* dst, long long count,
                            long long ncell, cudaStream_t s) {
    switch (storage) {
        case 1: return from_f64_t<float>(in, dst, count, ncell, s);
        case 4: return from_f64_t<__half>(in, dst, count, ncell, s);
        case 5: return from_f64_t<__nv_bfloat16>(in, dst, count, ncell, s);
        default:
            return cudaMemcpyAsync(dst, in, sizeof(double) * count, cudaMemcpyDeviceToDevice, s);
    }
}
cudaError_t launch_map(const Launch& L) {
    if (L.cp.np <= 0 || L.cp.kind == 0) return cudaSuccess;
    dim3 grid((L.map_ext[0] + 31) / 32, L.map_ext[1], L.map_ext[2] * L.cp.np);
    if (L.cp.kind == 2)
        k_map<2><<<grid, 32, 0, L.stream>>>(L.g, L.cp, L.parts, L.map, L.map_ext[0], L.map_ext[1],
                                            L.map_ext[2]);
    else
        k_map<1><<<grid, 32, 0, L.stream>>>(L.g, L.cp, L.parts, L.map, L.map_ext[0], L.map_ext[1],
                                            L.map_ext[2]);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Launch& L, int nsub, double* force_out, const double* charge) {
    if (L.cp.np <= 0) return cudaSuccess;
    k_finalize<<<L.cp.np, 256, 0, L.stream>>>(L.cp.np, near_blocks(L.box), L.partials, nsub,
                                               force_out, charge);
    return cudaGetLastError();
}
cudaError_t launch_rigid_body(const Launch& L, const double* force, double gx, double gy,
                              double gz, double dt, int wall_contact) {
    if (L.cp.np <= 0) return cudaSuccess;
    k_rigid<<<1, 32, 0, L.stream>>>(L.g, L.parts, L.parts_prev, L.cp.np, force, L.kd.rho0, gx, gy,
                                    gz, dt, wall_contact, L.status);
    return cudaGetLastError();
}
cudaError_t launch_regions(const Launch& L) {
    if (L.cp.np <= 0) return cudaSuccess;
    k_regions<<<1, 32, 0, L.stream>>>(L.g, L.parts, L.cp.np);
    return cudaGetLastError();
}


cudaError_t launch_batch_regions(BatchCase* cases, int n, cudaStream_t s) {
    k_batch_regions<<<(n + 63) / 64, 64, 0, s>>>(cases, n);
    return cudaGetLastError();
}
cudaError_t launch_batch_init(BatchCase* cases, int n, long long max_cells, cudaStream_t s) {
    dim3 grid((unsigned)((max_cells + 255) / 256), n, 1);
    k_batch_init<<<grid, 256, 0, s>>>(cases);
    return cudaGetLastError();
}
cudaError_t launch_batch_map(BatchCase* cases, BatchList l, long long total, cudaStream_t s) {
    if (l.n == 0 || total == 0) return cudaSuccess;
    k_batch_map<<<(unsigned)total, 32, 0, s>>>(cases, l);
    return cudaGetLastError();
}
cudaError_t launch_batch_near(BatchCase* cases, BatchList l, long long total, int sub,
                              int* status, cudaStream_t s) {
    if (l.n == 0 || total == 0) return cudaSuccess;
    k_batch_near<<<(unsigned)total, dim3(NEAR_BX, NEAR_BY, NEAR_BZ), 0, s>>>(cases, l, sub, status);
    return cudaGetLastError();
}
cudaError_t launch_batch_bulk(int mode, BatchCase* cases, BatchList l, long long total, int grid,
                              int* status, cudaStream_t s) {
    if (l.n == 0 || total == 0) return cudaSuccess;
    const unsigned gsz = (unsigned)(grid <= 0 || total < grid ? total : grid);
    if (mode == 3)
        k_batch_bulk<3><<<gsz, 256, 0, s>>>(cases, l, total, status);
    else
        k_batch_bulk<0><<<gsz, 256, 0, s>>>(cases, l, total, status);
    return cudaGetLastError();
}
cudaError_t launch_batch_swap(BatchCase* cases, BatchList l, cudaStream_t s) {
    if (l.n == 0) return cudaSuccess;
    k_batch_swap<<<(l.n + 63) / 64, 64, 0, s>>>(cases, l);
    return cudaGetLastError();
}
cudaError_t launch_batch_finalize(BatchCase* cases, int n, cudaStream_t s) {
    k_batch_finalize<<<n, 256, 0, s>>>(cases);
    return cudaGetLastError();
}
cudaError_t launch_batch_charge_total(BatchCase* cases, int n, cudaStream_t s) {
    k_batch_charge_total<<<(6 * n + 255) / 256, 256, 0, s>>>(cases, n);
    return cudaGetLastError();
}
cudaError_t launch_batch_rigid(BatchCase* cases, int n, int* status, cudaStream_t s) {
    k_batch_rigid<<<(n + 63) / 64, 64, 0, s>>>(cases, n, status);
    return cudaGetLastError();
}
// Device time stamp (the GPU's nanosecond global timer): end = 0 keeps it in
// p[0]; end = 1 adds the span since p[0] to p[1] and counts it in p[2].  One
// thread; launched on the stream of the work it brackets.
__global__ void k_stamp(unsigned long long* p, int end) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (!end) {
        p[0] = t;
    } else {
        p[1] += t - p[0];
        p[2] += 1;
    }
}
cudaError_t launch_stamp(unsigned long long* p, int end, cudaStream_t s) {
    k_stamp<<<1, 1, 0, s>>>(p, end);
    return cudaGetLastError();
}

cudaError_t launch_batch_refill(BatchCase* cases, BatchList l, long long total, int* status,
                                cudaStream_t s) {
    if (l.n == 0 || total == 0) return cudaSuccess;
    k_batch_refill<<<(unsigned)total, REFILL_THREADS, 0, s>>>(cases, l, status);
    return cudaGetLastError();
}
int batch_bulk_blocks_per_sm(int mode) {
    int nb = 0;
    if (mode == 3)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_bulk<3>, 256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_bulk<0>, 256, 0);
    return nb > 0 ? nb : 1;
}

}  // namespace lbmgpu
