// Device-side building blocks of the coupled D3Q19 sweep (sm_103a).
//
// Method: Rettinger & Ruede, arXiv:1702.04910, Sec. 2.  The sweep is the
// pull form of Eq. (1)-(2): each cell gathers the post-collision values of
// its upstream neighbours (stream, Eq. (2)), applies the wall / particle
// boundary conditions on the links it pulls across (Eq. (12), (14)),
// collides (Eq. (1) with Eq. (5) or (9), forcing Eq. (7); PSM Eq. (20)-(26))
// and writes its own 19 post-collision values.  The stored state between
// sweeps is therefore the post-collision field f~.
//
// Layout: structure of arrays f[q][z][y][x] (x fastest) so that a warp of
// 32 consecutive x reads and writes 32 consecutive elements per direction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_fixed.cuh"

namespace lbmgpu {

constexpr int NQ = 19;
constexpr int MAX_PARTICLES = 32;   // particle records staged in shared memory
constexpr int CELL_SLOTS = 2;       // objects that may touch one cell (Sec. 2.3, multi-object cells)
constexpr double NEAR_HALO = 2.0;   // cells around a sphere handled by the coupling kernels
// Distance a sphere surface keeps from an open z boundary (bc_z = 2): its
// near region (R + NEAR_HALO) then never contains a boundary plane, so only
// the plain pull needs the open-boundary rules.
constexpr double OPEN_MARGIN = 3.0;

// ---- D3Q19 velocity set (Sec. 2.1): rest, 6 axis, 12 diagonals in pairs ----
__host__ __device__ constexpr int cx(int q) {
    constexpr int t[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[q];
}
__host__ __device__ constexpr int cy(int q) {
    constexpr int t[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[q];
}
__host__ __device__ constexpr int cz(int q) {
    constexpr int t[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[q];
}
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ constexpr double wq(int q) {
    return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Particle record in device memory (160 B).  `reg` caches the near-particle
// region of the current state (see axis_range): per axis {cell start, cell
// count, tile start, tile count}, recomputed whenever the state changes.
struct DevParticle {
    double x[3], u[3], w[3];
    double d, r, rho, fixed;
    double pad;
    int reg[12];
    int pad2[2];
};

// Lattice geometry and tiling.  A tile is one thread block: tx * ty cells in
// one z plane.
struct Geom {
    int nx, ny, nz;
    int bc_z;           // 1: closed resting walls at z = 0 and z = nz;
                        // 2: inflow at z = 0, outflow at z = nz (Sec. 4.1)
    long long n;        // cells
    int tx, ty;         // tile extent in x, y (= block dims)
    int tz;             // z planes per tile (cells per thread along z in k_bulk)
    int ntx, nty, ntz;  // tiles per axis
    // open z boundaries (bc_z = 2)
    double uin[3];      // inflow velocity
    double rho_out;     // outflow density
    double rho0;        // reference density
    double fhalf[3];    // f_ext / (2 rho0): Eq. (8) velocity = j~/rho0 - fhalf
};

// Collision constants in the arithmetic type C.
template <typename C>
struct Coll {
    C lam_p, lam_m;   // lambda_+ = -1/tau, lambda_- from Eq. (11)
    C rho0, inv_rho0;
    C fx, fy, fz;     // f_ext
    int has_force;
    // folded constants of the pair update (see collide_fluid)
    C alpha, beta;    // 1 + (l+ + l-)/2, (l+ - l-)/2
    C hs, hd;         // (alpha + beta)/2 = (1 + l+)/2, (alpha - beta)/2 = (1 + l-)/2
    C c0;             // 1 + l+
    C m15r0;          // -3/2 / rho0 (multiplies j.j, j = rho0 U)
    C lpw[3];         // l+ w_k, k = rest, axis, diagonal
    C k1w[3];         // 9/2 l+ w_k / rho0 (multiplies (c.j)^2)
    C k2w[3];         // 3 l- w_k (multiplies c.j)
    C hw[3];          // 3 w_k / rho0 (times j.f_ext)
    C gq[10];         // 9 w_q (c_q . f_ext) / rho0, q = 1,3,...,17 (index (q-1)/2)
    C fq[10];         // 3 w_q (c_q . f_ext)
};

// Coupling constants (FP64: solid fractions, weights, forces).
struct Coupl {
    int kind;         // 0 none, 1 PSM, 2 MEM
    int variant;      // PSM: 0 M1B1, 1 M2B2, 2 M3B2; MEM: 0 BB, 1 CLI, 2 MR
    int np;
    int subsample;
    double tau;
    double rho0;
    double mr_cpc;    // MEM MR: -4 Lambda_- / (Lambda_- - 1/2), scale of the Eq. (15) correction
};

// ---------------------------------------------------------------------------
// Exactly rounded FP64 helpers for geometric predicates: these must give the
// same bits on every machine, so no contraction into fused multiply-adds.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Minimum-image separation along an axis of length L (periodic) or plain.
__device__ __forceinline__ double min_image(double d, double L, bool periodic) {
    if (!periodic) return d;
    double h = mul_rn(0.5, L);
    if (d > h) d = sub_rn(d, L);
    else if (d < -h) d = add_rn(d, L);
    return d;
}

__device__ __forceinline__ void separation(const Geom& g, double ax, double ay, double az,
                                           const DevParticle& P, double& dx, double& dy,
                                           double& dz) {
    dx = min_image(sub_rn(ax, P.x[0]), (double)g.nx, true);
    dy = min_image(sub_rn(ay, P.x[1]), (double)g.ny, true);
    dz = min_image(sub_rn(az, P.x[2]), (double)g.nz, !g.bc_z);
}

__device__ __forceinline__ double norm2_rn(double dx, double dy, double dz) {
    return add_rn(add_rn(mul_rn(dx, dx), mul_rn(dy, dy)), mul_rn(dz, dz));
}

// Point inside or on the sphere (MEM binary mapping, supersampling samples).
__device__ __forceinline__ bool point_inside(const Geom& g, const DevParticle& P, double px,
                                             double py, double pz) {
    double dx, dy, dz;
    separation(g, px, py, pz, P, dx, dy, dz);
    return norm2_rn(dx, dy, dz) <= mul_rn(P.r, P.r);
}

__device__ __forceinline__ bool cell_inside(const Geom& g, const DevParticle& P, int x, int y,
                                            int z) {
    return point_inside(g, P, x + 0.5, y + 0.5, z + 0.5);
}

// Owner of a cell under a particle set: 0 fluid, s+1 inside particle s.
__device__ __forceinline__ int cell_owner(const Geom& g, const DevParticle* parts, int np, int x,
                                          int y, int z) {
    for (int s = 0; s < np; ++s)
        if (cell_inside(g, parts[s], x, y, z)) return s + 1;
    return 0;
}

// Rigid-body velocity Eq. (13) at point p (minimum-image lever arm).
__device__ __forceinline__ void body_velocity(const Geom& g, const DevParticle& P, double px,
                                              double py, double pz, double& vx, double& vy,
                                              double& vz) {
    double rx, ry, rz;
    separation(g, px, py, pz, P, rx, ry, rz);
    vx = P.u[0] + (P.w[1] * rz - P.w[2] * ry);
    vy = P.u[1] + (P.w[2] * rx - P.w[0] * rz);
    vz = P.u[2] + (P.w[0] * ry - P.w[1] * rx);
}

// ---- near-particle regions -------------------------------------------------
// Along one axis, the cells whose centre lies within R + NEAR_HALO of the
// particle centre form a (possibly wrapped) cell range; the tiles holding
// them form a (possibly wrapped) tile range [lo, lo+len) mod nt.
struct AxisRange {
    int clo, clen;  // cell range start (wrapped) and length
    int tlo, tlen;  // tile range start (wrapped) and length
};

__device__ __forceinline__ int floor_div(int a, int b) {
    int q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}
__device__ __forceinline__ int wrap_i(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

__device__ inline AxisRange axis_range(double X, double R, int ncell, int T, int nt,
                                       bool periodic) {
    AxisRange r;
    // cells i with |i + 1/2 - X| <= R + halo  ->  i in [ceil(X-R-h-1/2), floor(X+R+h-1/2)]
    int lo = (int)ceil(X - R - NEAR_HALO - 0.5);
    int hi = (int)floor(X + R + NEAR_HALO - 0.5);
    if (!periodic) {
        lo = lo < 0 ? 0 : lo;
        hi = hi > ncell - 1 ? ncell - 1 : hi;
        r.clo = lo;
        r.clen = hi >= lo ? hi - lo + 1 : 0;
        if (r.clen == 0) {
            r.tlo = 0;
            r.tlen = 0;
            return r;
        }
        r.tlo = lo / T;
        r.tlen = hi / T - lo / T + 1;
        return r;
    }
    int len = hi - lo + 1;
    if (len >= ncell) {
        r.clo = 0;
        r.clen = ncell;
        r.tlo = 0;
        r.tlen = nt;
        return r;
    }
    int wlo = wrap_i(lo, ncell), whi = wrap_i(hi, ncell);
    r.clo = wlo;
    r.clen = len;
    int a = wlo / T, b = whi / T;
    r.tlo = a;
    r.tlen = wrap_i(b - a, nt) + 1;
    if (wlo > whi && a == b) r.tlen = nt;  // wrapped range re-entering its own tile
    return r;
}

// Offset of index i (in [0, n)) from the wrapped range start lo (in [0, n)).
__device__ __forceinline__ int range_off(int i, int lo, int n) {
    const int d = i - lo;
    return d < 0 ? d + n : d;
}

__device__ __forceinline__ bool in_range(int i, int lo, int len, int n) {
    return range_off(i, lo, n) < len;
}

// Whether the cell ranges [a, a + la) and [r, r + lr) of a periodic axis of
// n cells share a cell (a, r in [0, n); la, lr >= 1).
__device__ __forceinline__ bool spans_meet(int a, int la, int r, int lr, int n) {
    return range_off(a, r, n) < lr || range_off(r, a, n) < la;
}

struct NearRegion {
    AxisRange ax[3];
};

__device__ inline NearRegion near_region(const Geom& g, const DevParticle& P) {
    NearRegion nr;
    nr.ax[0] = axis_range(P.x[0], P.r, g.nx, g.tx, g.ntx, true);
    nr.ax[1] = axis_range(P.x[1], P.r, g.ny, g.ty, g.nty, true);
    nr.ax[2] = axis_range(P.x[2], P.r, g.nz, g.tz, g.ntz, !g.bc_z);
    return nr;
}

__device__ __forceinline__ bool tile_in_region(const Geom& g, const NearRegion& nr, int tx,
                                               int ty, int tz) {
    return in_range(tx, nr.ax[0].tlo, nr.ax[0].tlen, g.ntx) &&
           in_range(ty, nr.ax[1].tlo, nr.ax[1].tlen, g.nty) &&
           in_range(tz, nr.ax[2].tlo, nr.ax[2].tlen, g.ntz);
}

__device__ __forceinline__ bool cell_in_region(const Geom& g, const NearRegion& nr, int x, int y,
                                               int z) {
    return in_range(x, nr.ax[0].clo, nr.ax[0].clen, g.nx) &&
           in_range(y, nr.ax[1].clo, nr.ax[1].clen, g.ny) &&
           in_range(z, nr.ax[2].clo, nr.ax[2].clen, g.nz);
}

// Cache the region of P's current state in P.reg.
__device__ inline void store_region(const Geom& g, DevParticle& P) {
    NearRegion nr = near_region(g, P);
    for (int a = 0; a < 3; ++a) {
        P.reg[4 * a + 0] = nr.ax[a].clo;
        P.reg[4 * a + 1] = nr.ax[a].clen;
        P.reg[4 * a + 2] = nr.ax[a].tlo;
        P.reg[4 * a + 3] = nr.ax[a].tlen;
    }
}

__device__ __forceinline__ bool tile_in_reg(const Geom& g, const int* reg, int tx, int ty,
                                            int tz) {
    return in_range(tx, reg[2], reg[3], g.ntx) && in_range(ty, reg[6], reg[7], g.nty) &&
           in_range(tz, reg[10], reg[11], g.ntz);
}

__device__ __forceinline__ bool cell_in_reg(const Geom& g, const int* reg, int x, int y, int z) {
    return in_range(x, reg[0], reg[1], g.nx) && in_range(y, reg[4], reg[5], g.ny) &&
           in_range(z, reg[8], reg[9], g.nz);
}

// ---- pull (stream, Eq. (2)) ---------------------------------------------------
// Neighbour coordinates of a cell along -c_q (the upstream cell), with periodic
// wrap in x, y (and z if periodic).  zs is out of [0,nz) at a closed wall.
struct Nbr {
    int xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ Nbr make_nbr(const Geom& g, int x, int y, int z) {
    Nbr b;
    b.xm = x == 0 ? g.nx - 1 : x - 1;
    b.xp = x == g.nx - 1 ? 0 : x + 1;
    b.ym = y == 0 ? g.ny - 1 : y - 1;
    b.yp = y == g.ny - 1 ? 0 : y + 1;
    if (g.bc_z) {
        b.zm = z - 1;
        b.zp = z + 1;
    } else {
        b.zm = z == 0 ? g.nz - 1 : z - 1;
        b.zp = z == g.nz - 1 ? 0 : z + 1;
    }
    return b;
}

// Coordinates of x + k * c (k = +1 or -1) for a lattice direction q.
template <int Q>
__device__ __forceinline__ void shifted(const Nbr& b, int x, int y, int z, int sign, int& xs,
                                        int& ys, int& zs) {
    const int dx = sign * cx(Q), dy = sign * cy(Q), dz = sign * cz(Q);
    xs = dx > 0 ? b.xp : (dx < 0 ? b.xm : x);
    ys = dy > 0 ? b.yp : (dy < 0 ? b.ym : y);
    zs = dz > 0 ? b.zp : (dz < 0 ? b.zm : z);
}

__device__ __forceinline__ long long lin(const Geom& g, int x, int y, int z) {
    return (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
}

// ---- PDF storage --------------------------------------------------------------
// FP64 / FP32 store f_q itself.  The 16-bit formats store the shifted
// population f_q - w_q (rho0 = 1 reference state) so that the stored value is
// the small deviation from rest; loads add w_q back in FP32.
template <typename T>
struct PdfStore {
    template <typename C>
    __device__ __forceinline__ static C load(const T* p, int) {
        return (C)__ldg(p);
    }
    template <typename C>
    __device__ __forceinline__ static T save(C v, int) {
        return (T)v;
    }
};
template <>
struct PdfStore<__half> {
    template <typename C>
    __device__ __forceinline__ static C load(const __half* p, int q) {
        return (C)(__half2float(__ldg(p)) + (float)wq(q));
    }
    template <typename C>
    __device__ __forceinline__ static __half save(C v, int q) {
        return __float2half_rn((float)v - (float)wq(q));
    }
};
template <>
struct PdfStore<__nv_bfloat16> {
    template <typename C>
    __device__ __forceinline__ static C load(const __nv_bfloat16* p, int q) {
        return (C)(__bfloat162float(__ldg(p)) + (float)wq(q));
    }
    template <typename C>
    __device__ __forceinline__ static __nv_bfloat16 save(C v, int q) {
        return __float2bfloat16_rn((float)v - (float)wq(q));
    }
};

// Arithmetic type of the kernels that work on a storage type.
template <typename T> struct ComputeOf { using type = T; };
template <> struct ComputeOf<__half> { using type = float; };
template <> struct ComputeOf<__nv_bfloat16> { using type = float; };

template <typename T>
__device__ __forceinline__ double ld_pdf(const T* p, int q) {
    return PdfStore<T>::template load<double>(p, q);
}

// Linear-index offsets from a cell to its neighbours along each axis, with
// the periodic wrap folded in (z offsets 64-bit); zlo / zhi mark a closed
// wall just below / above the cell.
struct NbrOff {
    int dxm, dxp, dym, dyp;
    long long dzm, dzp;
    bool zlo, zhi;
};

__device__ __forceinline__ NbrOff make_off(const Geom& g, int x, int y, int z) {
    NbrOff o;
    o.dxm = x == 0 ? g.nx - 1 : -1;
    o.dxp = x == g.nx - 1 ? 1 - g.nx : 1;
    o.dym = y == 0 ? (g.ny - 1) * g.nx : -g.nx;
    o.dyp = y == g.ny - 1 ? (1 - g.ny) * g.nx : g.nx;
    const long long sz = (long long)g.nx * g.ny;
    o.zlo = g.bc_z && z == 0;
    o.zhi = g.bc_z && z == g.nz - 1;
    if (g.bc_z) {
        o.dzm = -sz;
        o.dzp = sz;
    } else {
        o.dzm = z == 0 ? (long long)(g.nz - 1) * sz : -sz;
        o.dzp = z == g.nz - 1 ? -(long long)(g.nz - 1) * sz : sz;
    }
    return o;
}

// Index offset of the upstream cell x - c_Q.
template <int Q>
__device__ __forceinline__ long long upstream_off(const NbrOff& o) {
    long long d = 0;
    if (cx(Q) > 0) d += o.dxm;
    else if (cx(Q) < 0) d += o.dxp;
    if (cy(Q) > 0) d += o.dym;
    else if (cy(Q) < 0) d += o.dyp;
    if (cz(Q) > 0) d += o.dzm;
    else if (cz(Q) < 0) d += o.dzp;
    return d;
}

// Plain pull of all 19 values for a fluid cell that has no particle link:
// periodic neighbours, halfway bounce-back at resting closed walls.
template <typename T, typename C, int Q>
__device__ __forceinline__ void pull_one(const T* __restrict__ src, const Geom& g,
                                         const NbrOff& o, long long idx, C (&f)[NQ]) {
    if ((cz(Q) > 0 && o.zlo) || (cz(Q) < 0 && o.zhi)) {
        f[Q] = PdfStore<T>::template load<C>(src + (long long)opp(Q) * g.n + idx, opp(Q));
    } else {
        f[Q] = PdfStore<T>::template load<C>(src + (long long)Q * g.n + idx + upstream_off<Q>(o), Q);
    }
}

template <typename T, typename C, int Q>
struct PullAll {
    __device__ __forceinline__ static void run(const T* __restrict__ src, const Geom& g,
                                               const NbrOff& o, long long idx, C (&f)[NQ]) {
        pull_one<T, C, Q>(src, g, o, idx, f);
        PullAll<T, C, Q + 1>::run(src, g, o, idx, f);
    }
};
template <typename T, typename C>
struct PullAll<T, C, NQ> {
    __device__ __forceinline__ static void run(const T* __restrict__, const Geom&, const NbrOff&,
                                               long long, C (&)[NQ]) {}
};

// Open z boundaries of the benchmark frame (bc_z = 2, Sec. 4.1).  PullAll has
// put the resting halfway bounce-back value f~_qbar(x) on every link that
// crosses z = 0 or z = nz.  Inflow (bottom): the moving-wall term of Eq. (12)
// with u_in is added, f_q = f~_qbar(x) + 2 w_q rho0 (c_q . u_in) / c_s^2.
// Outflow (top): f_q = -f~_qbar(x) + 2 f_eq,+_q(rho_out, u(x)), f_eq,+ the
// even part of Eq. (3), u(x) the Eq. (8) velocity of the cell (its
// post-collision momentum j~ = j + f_ext, so u = j~/rho0 - f_ext/(2 rho0)).
template <typename T, typename C>
__device__ __forceinline__ void open_boundaries(const T* __restrict__ src, const Geom& g,
                                                const NbrOff& o, long long idx, C (&f)[NQ]) {
    if (o.zlo) {
#pragma unroll
        for (int q = 1; q < NQ; ++q) {
            if (cz(q) <= 0) continue;
            const double cu = cx(q) * g.uin[0] + cy(q) * g.uin[1] + cz(q) * g.uin[2];
            f[q] = f[q] + (C)(6.0 * wq(q) * g.rho0 * cu);
        }
    }
    if (o.zhi) {
        double j[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int q = 1; q < NQ; ++q) {
            const double v = ld_pdf(src + (long long)q * g.n + idx, q);
            j[0] += v * cx(q);
            j[1] += v * cy(q);
            j[2] += v * cz(q);
        }
        double u[3];
        for (int a = 0; a < 3; ++a) u[a] = j[a] / g.rho0 - g.fhalf[a];
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
        for (int q = 1; q < NQ; ++q) {
            if (cz(q) >= 0) continue;
            const double cu = cx(q) * u[0] + cy(q) * u[1] + cz(q) * u[2];
            const double feq_even = wq(q) * (g.rho_out + g.rho0 * (4.5 * cu * cu - 1.5 * uu));
            f[q] = (C)(2.0 * feq_even - (double)f[q]);
        }
    }
}

template <typename T, typename C>
__device__ __forceinline__ void pull_plain(const T* __restrict__ src, const Geom& g, int x, int y,
                                           int z, long long idx, C (&f)[NQ]) {
    const NbrOff o = make_off(g, x, y, z);
    PullAll<T, C, 0>::run(src, g, o, idx, f);
    if (g.bc_z == 2 && (o.zlo || o.zhi)) open_boundaries(src, g, o, idx, f);
}

template <typename T, typename C>
__device__ __forceinline__ void load_own(const T* __restrict__ src, const Geom& g, long long idx,
                                         C (&f)[NQ]) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) f[q] = PdfStore<T>::template load<C>(src + (long long)q * g.n + idx, q);
}

template <typename T, typename C>
__device__ __forceinline__ void store_own(T* __restrict__ dst, const Geom& g, long long idx,
                                          const C (&f)[NQ]) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) dst[(long long)q * g.n + idx] = PdfStore<T>::template save<C>(f[q], q);
}

// ---- moments Eq. (4) ---------------------------------------------------------
template <typename C>
__device__ __forceinline__ void moments(const C (&f)[NQ], const Coll<C>& k, C& rho, C& ux, C& uy,
                                        C& uz) {
    C s1 = f[1] + f[2], s3 = f[3] + f[4], s5 = f[5] + f[6], s7 = f[7] + f[8];
    C s9 = f[9] + f[10], s11 = f[11] + f[12], s13 = f[13] + f[14], s15 = f[15] + f[16];
    C s17 = f[17] + f[18];
    rho = f[0] + ((s1 + s3) + (s5 + s7)) + ((s9 + s11) + (s13 + s15)) + s17;
    C d1 = f[1] - f[2], d3 = f[3] - f[4], d5 = f[5] - f[6], d7 = f[7] - f[8];
    C d9 = f[9] - f[10], d11 = f[11] - f[12], d13 = f[13] - f[14], d15 = f[15] - f[16];
    C d17 = f[17] - f[18];
    ux = ((d1 + d7) + (d9 + d11) + d13) * k.inv_rho0;
    uy = ((d3 + d7) - (d9 - d15) + d17) * k.inv_rho0;
    uz = ((d5 + d11) - (d13 - d15) - d17) * k.inv_rho0;
}

// Density and momentum j = rho0 U of Eq. (4) (the collision works with j and
// constants that carry the 1/rho0: three products fewer per cell).
template <typename C>
__device__ __forceinline__ void moments_j(const C (&f)[NQ], C& rho, C& jx, C& jy, C& jz) {
    C s1 = f[1] + f[2], s3 = f[3] + f[4], s5 = f[5] + f[6], s7 = f[7] + f[8];
    C s9 = f[9] + f[10], s11 = f[11] + f[12], s13 = f[13] + f[14], s15 = f[15] + f[16];
    C s17 = f[17] + f[18];
    rho = f[0] + ((s1 + s3) + (s5 + s7)) + ((s9 + s11) + (s13 + s15)) + s17;
    C d1 = f[1] - f[2], d3 = f[3] - f[4], d5 = f[5] - f[6], d7 = f[7] - f[8];
    C d9 = f[9] - f[10], d11 = f[11] - f[12], d13 = f[13] - f[14], d15 = f[15] - f[16];
    C d17 = f[17] - f[18];
    jx = (d1 + d7) + (d9 + d11) + d13;
    jy = (d3 + d7) - (d9 - d15) + d17;
    jz = (d5 + d11) - (d13 - d15) - d17;
}

// ---- fluid collision Eq. (1) with TRT Eq. (9)-(10) (BGK: lambda_- = lambda_+)
// and forcing Eq. (7), in place, written per opposite pair (q, qbar):
//   f^eq,+ = w (rho + rho0 (9/2 (c.U)^2 - 3/2 U.U)),  f^eq,- = 3 w rho0 c.U,
//   F^+ = w (9 (c.U)(c.f) - 3 U.f),                   F^- = 3 w c.f.
// The per-pair update is written with the relaxation folded in:
//   f_q'    = alpha f_q    + beta f_qbar - (P + M)
//   f_qbar' = alpha f_qbar + beta f_q    - (P - M)
// with P = l+ f^eq,+ - F^+ and M = l- f^eq,- - F^-, which expands
// f_q + l+ (f_q^+ - f^eq,+) + l- (f_q^- - f^eq,-) + F_q exactly.
// Arithmetic whose products cost far more than its sums (the 64-bit fixed
// point) takes the pair update in sum / difference form,
//   f_q' = hs (f_q + f_qbar) + hd (f_q - f_qbar) - (P + M),
//   f_qbar' = hs (f_q + f_qbar) - hd (f_q - f_qbar) - (P - M):
// two products per pair instead of four (PairSumDiff, lbm_fixed.cuh).
// C is the arithmetic type, KT the type of the constants (C itself, or float
// for the packed f2: C(k.x) broadcasts a constant to both lanes).
template <typename C, int Q, int K, bool FORCE, typename KT>
__device__ __forceinline__ void trt_pair(C (&f)[NQ], C cu, const C (&bw)[3], const Coll<KT>& k) {
    constexpr int QB = Q + 1;
    C P = FORCE ? fma(C(k.k1w[K]), cu * cu, fma(C(-k.gq[(Q - 1) / 2]), cu, bw[K]))
                : fma(C(k.k1w[K]), cu * cu, bw[K]);
    C M = FORCE ? fma(C(k.k2w[K]), cu, C(-k.fq[(Q - 1) / 2])) : C(k.k2w[K]) * cu;
    const C a = f[Q], b = f[QB];
    if constexpr (PairSumDiff<C>::value) {
        const C sp = k.hs * (a + b), sd = k.hd * (a - b);
        f[Q] = (sp + sd) - (P + M);
        f[QB] = (sp - sd) - (P - M);
    } else {
        f[Q] = fma(C(k.alpha), a, fma(C(k.beta), b, -(P + M)));
        f[QB] = fma(C(k.alpha), b, fma(C(k.beta), a, -(P - M)));
    }
}

// Sum / difference pair update with P given (see trt_pair).
template <typename C, int Q, int K>
__device__ __forceinline__ void trt_pair_sd(C (&f)[NQ], C cu, C P, const Coll<C>& k) {
    constexpr int QB = Q + 1;
    const C M = k.k2w[K] * cu;
    const C a = f[Q], b = f[QB];
    const C sp = k.hs * (a + b), sd = k.hd * (a - b);
    f[Q] = (sp + sd) - (P + M);
    f[QB] = (sp - sd) - (P - M);
}

// Two FP32 lanes in one register pair, for the Blackwell packed f32x2
// add / multiply / FMA (one instruction for both lanes, each lane rounded as
// the scalar operation).  The 16-bit pair sweep keeps its two cells in the two
// lanes; constants are broadcast with f2(c).
struct f2 {
    float2 v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ explicit f2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ explicit f2(float2 x) : v(x) {}
};
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }

// Fluid health: the density of Eq. (4) of a cell must be finite and
// positive.  Bit tests on the integer pipes (no FP64 instruction): a value
// outside (0, +inf) -- zero, negative, infinite or NaN -- is reported.  (The
// float-float form is in lbm_dfloat.cuh; overloads are found at
// instantiation.)
__device__ __forceinline__ bool density_bad(double r) {
    return (unsigned long long)__double_as_longlong(r) - 1ull >= 0x7FEFFFFFFFFFFFFFull;
}
__device__ __forceinline__ bool density_bad(float r) {
    return __float_as_uint(r) - 1u >= 0x7F7FFFFFu;
}
// packed pair: bit 0 for lane x, bit 1 for lane y
__device__ __forceinline__ unsigned density_bad(f2 r) {
    return (density_bad(r.v.x) ? 1u : 0u) | (density_bad(r.v.y) ? 2u : 0u);
}
// fixed point cannot hold NaN (the conversion from FP64 turns a non-finite
// value into 0); a saturated conversion or a wrapped sum shows as a density
// outside (0, 16)
__device__ __forceinline__ bool density_bad(fx64 r) {
    return !(r.v > 0 && r.v < (16LL << FX_SHIFT));
}

// Returns true when the cell's density is not finite and positive.
// SHIFTED: f holds the shifted populations f_q - w_q, whose sum is rho - 1.
// Written in j = rho0 U (ux, uy, uz below hold j); the constants k1w, k2w,
// m15r0, hw and gq carry the powers of 1/rho0 that U would bring.
// KT: type of the constants (see trt_pair).  The result is density_bad's:
// a bool, or a lane mask for the packed f2.
template <typename C, bool FORCE, bool SHIFTED, typename KT>
__device__ __forceinline__ auto collide_fluid_t(C (&f)[NQ], const Coll<KT>& k) {
    C rho, ux, uy, uz;
    moments_j(f, rho, ux, uy, uz);
    const auto bad = SHIFTED ? density_bad(rho + C(1)) : density_bad(rho);
    if constexpr (PairSumDiff<C>::value && !FORCE) {
        // products shared between pairs: with t_a = k1w_diag u_a^2 and
        // c_ab = k1w_axis u_a u_b (k1w_axis = 2 k1w_diag), the quadratic term
        // of P is 2 t_a on an axis pair and t_a + t_b +- c_ab on a diagonal one
        const C xx = ux * ux, yy = uy * uy, zz = uz * uz;
        const C base = fma(k.m15r0, (xx + yy) + zz, rho);
        C bw[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) bw[c] = k.lpw[c] * base;
        const C tx = k.k1w[2] * xx, ty = k.k1w[2] * yy, tz = k.k1w[2] * zz;
        const C cxy = k.k1w[1] * (ux * uy), cxz = k.k1w[1] * (ux * uz), cyz = k.k1w[1] * (uy * uz);
        f[0] = fma(k.c0, f[0], -bw[0]);
        trt_pair_sd<C, 1, 1>(f, ux, (tx + tx) + bw[1], k);
        trt_pair_sd<C, 3, 1>(f, uy, (ty + ty) + bw[1], k);
        trt_pair_sd<C, 5, 1>(f, uz, (tz + tz) + bw[1], k);
        trt_pair_sd<C, 7, 2>(f, ux + uy, ((tx + ty) + cxy) + bw[2], k);
        trt_pair_sd<C, 9, 2>(f, ux - uy, ((tx + ty) - cxy) + bw[2], k);
        trt_pair_sd<C, 11, 2>(f, ux + uz, ((tx + tz) + cxz) + bw[2], k);
        trt_pair_sd<C, 13, 2>(f, ux - uz, ((tx + tz) - cxz) + bw[2], k);
        trt_pair_sd<C, 15, 2>(f, uy + uz, ((ty + tz) + cyz) + bw[2], k);
        trt_pair_sd<C, 17, 2>(f, uy - uz, ((ty + tz) - cyz) + bw[2], k);
        return bad;
    }
    const C uu = fma(ux, ux, fma(uy, uy, uz * uz));
    const C base = fma(C(k.m15r0), uu, rho);
    C bw[3];
    if (FORCE) {
        const C uf = fma(ux, C(k.fx), fma(uy, C(k.fy), uz * C(k.fz)));
#pragma unroll
        for (int c = 0; c < 3; ++c) bw[c] = fma(C(k.lpw[c]), base, C(k.hw[c]) * uf);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) bw[c] = C(k.lpw[c]) * base;
    }
    f[0] = fma(C(k.c0), f[0], -bw[0]);
    trt_pair<C, 1, 1, FORCE>(f, ux, bw, k);
    trt_pair<C, 3, 1, FORCE>(f, uy, bw, k);
    trt_pair<C, 5, 1, FORCE>(f, uz, bw, k);
    trt_pair<C, 7, 2, FORCE>(f, ux + uy, bw, k);
    trt_pair<C, 9, 2, FORCE>(f, ux - uy, bw, k);
    trt_pair<C, 11, 2, FORCE>(f, ux + uz, bw, k);
    trt_pair<C, 13, 2, FORCE>(f, ux - uz, bw, k);
    trt_pair<C, 15, 2, FORCE>(f, uy + uz, bw, k);
    trt_pair<C, 17, 2, FORCE>(f, uy - uz, bw, k);
    return bad;
}

// Fluid collision Eq. (1) with TRT Eq. (9)-(10) (BGK: lambda_- = lambda_+)
// and forcing Eq. (7), in place.  Returns true when the cell's density is
// not finite and positive (density_bad).  SHIFTED: f holds f_q - w_q (the
// 16-bit storage's populations, collided as they are).
template <typename C, bool SHIFTED = false, typename KT>
__device__ __forceinline__ auto collide_fluid(C (&f)[NQ], const Coll<KT>& k) {
    if (k.has_force) return collide_fluid_t<C, true, SHIFTED>(f, k);
    return collide_fluid_t<C, false, SHIFTED>(f, k);
}

// Collision operator values C_q (Eq. (5)/(9)) and forcing F_q (Eq. (7)) as
// separate arrays, for the PSM blend Eq. (26).  Also returns rho and U.
template <typename C>
__device__ inline void fluid_operator(const C (&f)[NQ], const Coll<C>& k, C (&Cf)[NQ],
                                      C (&Fq)[NQ], C& rho, C& ux, C& uy, C& uz) {
    moments(f, k, rho, ux, uy, uz);
    C uu = ux * ux + uy * uy + uz * uz;
    C base = rho - (C)1.5 * k.rho0 * uu;
    C uf = ux * k.fx + uy * k.fy + uz * k.fz;
    Cf[0] = k.lam_p * (f[0] - (C)(1.0 / 3.0) * base);
    Fq[0] = (C)(1.0 / 3.0) * ((C)-3 * uf);
#pragma unroll
    for (int q = 1; q < NQ; q += 2) {
        const C w = (C)wq(q);
        C cu = (C)cx(q) * ux + (C)cy(q) * uy + (C)cz(q) * uz;
        C cf = (C)cx(q) * k.fx + (C)cy(q) * k.fy + (C)cz(q) * k.fz;
        C fs = f[q] + f[q + 1], fd = f[q] - f[q + 1];
        C eqs = w * (base + (C)4.5 * k.rho0 * cu * cu);
        C eqd = (C)3 * w * k.rho0 * cu;
        C cs = k.lam_p * ((C)0.5 * fs - eqs);
        C cd = k.lam_m * ((C)0.5 * fd - eqd);
        Cf[q] = cs + cd;
        Cf[q + 1] = cs - cd;
        C fsym = w * ((C)9 * cu * cf - (C)3 * uf);
        C fanti = (C)3 * w * cf;
        Fq[q] = fsym + fanti;
        Fq[q + 1] = fsym - fanti;
    }
}

// Equilibrium Eq. (3) for all q at density rho and velocity (vx, vy, vz).
template <typename C>
__device__ __forceinline__ void equilibrium(C rho, C vx, C vy, C vz, C rho0, C (&e)[NQ]) {
    C base = rho - (C)1.5 * rho0 * (vx * vx + vy * vy + vz * vz);
    e[0] = (C)(1.0 / 3.0) * base;
#pragma unroll
    for (int q = 1; q < NQ; q += 2) {
        const C w = (C)wq(q);
        C cu = (C)cx(q) * vx + (C)cy(q) * vy + (C)cz(q) * vz;
        C s = w * (base + (C)4.5 * rho0 * cu * cu);
        C d = (C)3 * w * rho0 * cu;
        e[q] = s + d;
        e[q + 1] = s - d;
    }
}

// ---- PSM solid fraction: n^3 supersampling (Sec. 2.3) -----------------------
// Number of the n^3 sub-cell samples at ((i + 1/2)/n, ...) inside the sphere.
// Cells wholly inside the sphere give n^3 and cells whose box misses the
// sphere give 0 without sampling; both short-cuts agree exactly with the
// sampled count (samples lie at least 1/(2n) inside the cell, far beyond
// rounding).  For n a power of two the sample offsets (2i+1) * (1/(2n)) are
// the same doubles as (i + 1/2)/n, without a division.
__device__ inline int solid_count(const Geom& g, const DevParticle& P, int x, int y, int z,
                                  int n) {
    double dx, dy, dz;
    separation(g, x + 0.5, y + 0.5, z + 0.5, P, dx, dy, dz);
    double ax = fabs(dx), ay = fabs(dy), az = fabs(dz);
    double nxd = fmax(ax - 0.5, 0.0), nyd = fmax(ay - 0.5, 0.0), nzd = fmax(az - 0.5, 0.0);
    double R2 = mul_rn(P.r, P.r);
    if (norm2_rn(nxd, nyd, nzd) > R2 * (1.0 + 1e-12) + 1e-9) return 0;
    double fxd = ax + 0.5, fyd = ay + 0.5, fzd = az + 0.5;
    if (norm2_rn(fxd, fyd, fzd) < R2 * (1.0 - 1e-12) - 1e-9) return n * n * n;
    const bool pow2 = (n & (n - 1)) == 0;
    const double h = 0.5 / n;  // exact for n a power of two
    const double X = x, Y = y, Z = z;
    int inside = 0;
    for (int k = 0; k < n; ++k) {
        const double pz = Z + (pow2 ? (2 * k + 1) * h : (k + 0.5) / n);
        for (int j = 0; j < n; ++j) {
            const double py = Y + (pow2 ? (2 * j + 1) * h : (j + 0.5) / n);
            for (int i = 0; i < n; ++i) {
                const double px = X + (pow2 ? (2 * i + 1) * h : (i + 0.5) / n);
                inside += point_inside(g, P, px, py, pz) ? 1 : 0;
            }
        }
    }
    return inside;
}

// solid_count with the n^3 samples spread over the 32 lanes of a warp: every
// lane passes the same cell; all lanes must call it (warp-synchronous).  Same
// predicate and the same integer count as solid_count.
__device__ inline int solid_count_warp(const Geom& g, const DevParticle& P, int x, int y, int z,
                                       int n, int lane) {
    const bool pow2 = (n & (n - 1)) == 0;
    const double h = 0.5 / n;
    const double X = x, Y = y, Z = z;
    int inside = 0;
    for (int s = lane; s < n * n * n; s += 32) {
        const int i = s % n, j = (s / n) % n, k = s / (n * n);
        const double pz = Z + (pow2 ? (2 * k + 1) * h : (k + 0.5) / n);
        const double py = Y + (pow2 ? (2 * j + 1) * h : (j + 0.5) / n);
        const double px = X + (pow2 ? (2 * i + 1) * h : (i + 0.5) / n);
        inside += point_inside(g, P, px, py, pz) ? 1 : 0;
    }
    return __reduce_add_sync(0xffffffffu, inside);
}

// The quick part of solid_count: 0 or n^3 for cells wholly outside / inside
// the sphere, -1 for cells that need the samples.
__device__ inline int solid_count_quick(const Geom& g, const DevParticle& P, int x, int y, int z,
                                        int n) {
    double dx, dy, dz;
    separation(g, x + 0.5, y + 0.5, z + 0.5, P, dx, dy, dz);
    double ax = fabs(dx), ay = fabs(dy), az = fabs(dz);
    double nxd = fmax(ax - 0.5, 0.0), nyd = fmax(ay - 0.5, 0.0), nzd = fmax(az - 0.5, 0.0);
    double R2 = mul_rn(P.r, P.r);
    if (norm2_rn(nxd, nyd, nzd) > R2 * (1.0 + 1e-12) + 1e-9) return 0;
    double fxd = ax + 0.5, fyd = ay + 0.5, fzd = az + 0.5;
    if (norm2_rn(fxd, fyd, fzd) < R2 * (1.0 - 1e-12) - 1e-9) return n * n * n;
    return -1;
}

__device__ inline double solid_fraction(const Geom& g, const DevParticle& P, int x, int y, int z,
                                        int n) {
    return (double)solid_count(g, P, x, y, z, n) / ((double)n * n * n);
}

// Per-step geometry map of a particle's near region (see k_map): MEM owner
// (0 fluid, s+1 inside particle s) or PSM supersample count of that particle.
struct GeoMap {
    const unsigned short* map;  // [particle][z][y][x] over the region box
    int ex, ey, ez;             // box extents (cells)
};

// Region offsets of (x,y,z) in particle s's region; false if outside it.
__device__ __forceinline__ bool region_offsets(const Geom& g, const int* r, int x, int y, int z,
                                               int& ox, int& oy, int& oz) {
    ox = range_off(x, r[0], g.nx);
    oy = range_off(y, r[4], g.ny);
    oz = range_off(z, r[8], g.nz);
    return ox < r[1] && oy < r[5] && oz < r[9];
}

// Offsets outside the map read as 0 (fluid / uncovered) without touching
// memory; callers only pass offsets inside a region box.
__device__ __forceinline__ unsigned short map_at(const GeoMap& m, int s, int ox, int oy, int oz) {
    if (s < 0 || s >= MAX_PARTICLES || ox < 0 || ox >= m.ex || oy < 0 || oy >= m.ey || oz < 0 ||
        oz >= m.ez)
        return 0;
    return __ldg(m.map + (((long long)s * m.ez + oz) * m.ey + oy) * m.ex + ox);
}

// MEM owner of a cell from the map (0 fluid, s+1 inside particle s).
__device__ __forceinline__ int mapped_owner(const Geom& g, const DevParticle* parts, int np,
                                            const GeoMap& m, int x, int y, int z) {
    for (int s = 0; s < np; ++s) {
        int ox, oy, oz;
        if (region_offsets(g, parts[s].reg, x, y, z, ox, oy, oz)) return map_at(m, s, ox, oy, oz);
    }
    return 0;
}

// ---- MEM link geometry ---------------------------------------------------------
// delta: smallest root t of |x + t c - X| = R, clamped to [0, 1].
__device__ inline double link_delta(const Geom& g, const DevParticle& P, double px, double py,
                                    double pz, int ccx, int ccy, int ccz) {
    double dx, dy, dz;
    separation(g, px, py, pz, P, dx, dy, dz);
    double a = (double)(ccx * ccx + ccy * ccy + ccz * ccz);
    double b = dx * ccx + dy * ccy + dz * ccz;
    double c = (dx * dx + dy * dy + dz * dz) - P.r * P.r;
    double disc = b * b - a * c;
    if (disc < 0.0) disc = 0.0;
    double t = (-b - sqrt(disc)) / a;
    return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
}

// ---- block reductions (FP64) --------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace lbmgpu
