// Learned force correction: the near-surface feature stencil of a particle,
// a small MLP (512 -> 64 -> 64 -> 6, tanh) with hand-written forward,
// backward and Adam kernels, and its use inside the coupled step
// (declarations and contracts in include/lbm_gb300.h).
//
// The paper has no learned component; this is an extension that corrects the
// hydrodynamic force and torque of a coarsely resolved sphere (Sec. 4 studies
// how that force converges with the resolution D) towards a finely resolved
// run of the same method.
//
// Features of particle p (all FP32, computed in FP64):
//   [0,125)    solid indicator at a 5 x 5 x 5 grid of points around the
//              centre X_p, spacing h = (R + 2) / 2 (the grid spans the sphere
//              and its two-cell near-surface layer), trilinear from the cell
//              centres: PSM total solid fraction (min(sum eps_s, 1)), MEM
//              1 for a solid cell, 0 for a fluid cell (both read from the
//              step's geometry map);
//   [125,500)  (u - U_p) / u_ref at the same points, x then y then z blocks;
//              u = j~ / rho0 of the stored post-collision PDFs, the body
//              velocity in a MEM solid cell, 0 beyond a closed wall;
//   [500,512)  U_p / u_ref, Omega_p R / u_ref, F / (rho0 u_ref^2 D^2),
//              T / (rho0 u_ref^2 D^3) (F, T: this step's hydrodynamic force).
// Outputs: the correction (dF, dT) in the same units as the last two blocks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbm_gb300.h"
#include "lbm_launch.h"

using namespace lbmgpu;

namespace lbmgpu {

constexpr int FIN = LBM_MLP_IN, FH = LBM_MLP_HIDDEN, FOUT = LBM_MLP_OUT;
constexpr int NSTEN = 5, NPTS = NSTEN * NSTEN * NSTEN;
// parameter offsets (weights stored [in][out]: output index fastest)
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + FIN * FH;
constexpr int OFF_W2 = OFF_B1 + FH;
constexpr int OFF_B2 = OFF_W2 + FH * FH;
constexpr int OFF_W3 = OFF_B2 + FH;
constexpr int OFF_B3 = OFF_W3 + FH * FOUT;
constexpr int NPARAM = OFF_B3 + FOUT;
static_assert(NPARAM == LBM_MLP_PARAMS, "parameter count");
// normalisation block: input mean [FIN], input 1/std [FIN], output scale [FOUT]
constexpr int NORM_MU = 0, NORM_IS = FIN, NORM_OS = 2 * FIN, NNORM = 2 * FIN + FOUT;

// ---------------------------------------------------------------------------
// feature stencil: one block per particle, one thread per grid point
template <typename T>
__global__ void __launch_bounds__(128)
    k_features(const T* __restrict__ state, Geom g, Coupl cp, const DevParticle* __restrict__ parts,
               GeoMap gm, const double* __restrict__ force, double u_ref, float* __restrict__ feat) {
    __shared__ DevParticle sp[MAX_PARTICLES];
    const int nd = cp.np * (int)(sizeof(DevParticle) / sizeof(double));
    for (int i = threadIdx.x; i < nd; i += blockDim.x)
        reinterpret_cast<double*>(sp)[i] = reinterpret_cast<const double*>(parts)[i];
    __syncthreads();
    const int p = blockIdx.x;
    const DevParticle& P = sp[p];
    float* out = feat + (long long)p * FIN;
    const int s = threadIdx.x;
    if (s < NPTS) {
        const int i = s % NSTEN, j = (s / NSTEN) % NSTEN, k = s / (NSTEN * NSTEN);
        const double h = 0.5 * (P.r + NEAR_HALO);
        const double pos[3] = {P.x[0] + (i - 2) * h, P.x[1] + (j - 2) * h, P.x[2] + (k - 2) * h};
        int base[3];
        double fr[3];
        for (int a = 0; a < 3; ++a) {
            const double c = pos[a] - 0.5;  // cell-centre coordinate
            const double fl = floor(c);
            base[a] = (int)fl;
            fr[a] = c - fl;
        }
        const double n3 = (double)cp.subsample * cp.subsample * cp.subsample;
        double eps = 0.0, u[3] = {0.0, 0.0, 0.0};
        for (int corner = 0; corner < 8; ++corner) {
            const int d[3] = {corner & 1, (corner >> 1) & 1, (corner >> 2) & 1};
            double w = 1.0;
            for (int a = 0; a < 3; ++a) w *= d[a] ? fr[a] : 1.0 - fr[a];
            const int X = wrap_i(base[0] + d[0], g.nx), Y = wrap_i(base[1] + d[1], g.ny);
            int Z = base[2] + d[2];
            if (g.bc_z) {
                if (Z < 0 || Z >= g.nz) continue;  // beyond a resting wall: eps 0, u 0
            } else {
                Z = wrap_i(Z, g.nz);
            }
            const double xc = X + 0.5, yc = Y + 0.5, zc = Z + 0.5;
            double e = 0.0, v[3] = {0.0, 0.0, 0.0};
            int own = 0;
            // the step's geometry map (cells outside every region box are
            // fluid / uncovered)
            if (cp.kind == 2) {
                own = mapped_owner(g, sp, cp.np, gm, X, Y, Z);
                e = own ? 1.0 : 0.0;
            } else if (cp.kind == 1) {
                for (int q = 0; q < cp.np; ++q) {
                    int ox, oy, oz;
                    if (region_offsets(g, sp[q].reg, X, Y, Z, ox, oy, oz)) e += map_at(gm, q, ox, oy, oz) / n3;
                }
                e = e < 1.0 ? e : 1.0;
            }
            if (own) {
                body_velocity(g, sp[own - 1], xc, yc, zc, v[0], v[1], v[2]);
            } else {
                const long long idx = lin(g, X, Y, Z);
                for (int q = 0; q < NQ; ++q) {
                    const double f = ld_pdf(state + (long long)q * g.n + idx, q);
                    v[0] += f * cx(q);
                    v[1] += f * cy(q);
                    v[2] += f * cz(q);
                }
                for (int a = 0; a < 3; ++a) v[a] /= cp.rho0;
            }
            eps += w * e;
            for (int a = 0; a < 3; ++a) u[a] += w * v[a];
        }
        out[s] = (float)eps;
        for (int a = 0; a < 3; ++a) out[NPTS * (1 + a) + s] = (float)((u[a] - P.u[a]) / u_ref);
    }
    if (s == 0) {
        const double D = P.d, fs = cp.rho0 * u_ref * u_ref * D * D, ts = fs * D;
        const double* F = force + 6 * p;
        for (int a = 0; a < 3; ++a) {
            out[4 * NPTS + a] = (float)(P.u[a] / u_ref);
            out[4 * NPTS + 3 + a] = (float)(P.w[a] * P.r / u_ref);
            out[4 * NPTS + 6 + a] = (float)(F[a] / fs);
            out[4 * NPTS + 9 + a] = (float)(F[3 + a] / ts);
        }
    }
}

// ---------------------------------------------------------------------------
// MLP forward: one 64-thread block per sample.  Inputs are normalised on
// load, x^ = (x - mu) / sigma; the network output y^ is kept (normalised)
// and y = y^ * out_scale returned.  H1, H2 may be null (inference).
// With clip > 0 a sample with any |x^_i| > clip (outside the training data)
// gets y = 0: the caller's plain force stands.
__global__ void __launch_bounds__(FH)
    k_mlp_forward(const float* __restrict__ P, const float* __restrict__ norm,
                  const float* __restrict__ X, int n, float* __restrict__ H1,
                  float* __restrict__ H2, float* __restrict__ Yn, float* __restrict__ Y,
                  float clip) {
    __shared__ float xs[FIN], h1[FH], h2[FH];
    const int smp = blockIdx.x, u = threadIdx.x;
    if (smp >= n) return;
    const float* x = X + (long long)smp * FIN;
    int out_of_range = 0;
    for (int i = u; i < FIN; i += FH) {
        const float v = (x[i] - norm[NORM_MU + i]) * norm[NORM_IS + i];
        xs[i] = v;
        out_of_range |= clip > 0.0f && !(fabsf(v) <= clip);
    }
    if (__syncthreads_or(out_of_range)) {
        if (u < FOUT) {
            if (Yn) Yn[(long long)smp * FOUT + u] = 0.0f;
            if (Y) Y[(long long)smp * FOUT + u] = 0.0f;
        }
        return;
    }
    float a = P[OFF_B1 + u];
    for (int i = 0; i < FIN; ++i) a = fmaf(P[OFF_W1 + i * FH + u], xs[i], a);
    const float t1 = tanhf(a);
    h1[u] = t1;
    if (H1) H1[(long long)smp * FH + u] = t1;
    __syncthreads();
    a = P[OFF_B2 + u];
    for (int v = 0; v < FH; ++v) a = fmaf(P[OFF_W2 + v * FH + u], h1[v], a);
    const float t2 = tanhf(a);
    h2[u] = t2;
    if (H2) H2[(long long)smp * FH + u] = t2;
    __syncthreads();
    if (u < FOUT) {
        a = P[OFF_B3 + u];
        for (int v = 0; v < FH; ++v) a = fmaf(P[OFF_W3 + v * FOUT + u], h2[v], a);
        if (Yn) Yn[(long long)smp * FOUT + u] = a;
        if (Y) Y[(long long)smp * FOUT + u] = a * norm[NORM_OS + u];
    }
}

// Backward deltas of the loss L = 1/(2n) sum_s sum_k w_k (y^_sk - t_sk / os_k)^2,
// w_k = (os_k / max_j os_j)^2 (each output's error in the units of the
// largest target), one 64-thread block per sample: D3 = dL/dz3, D2 = dL/dz2,
// D1 = dL/dz1 (z: pre-activations), and the sample's loss term.
__global__ void __launch_bounds__(FH)
    k_mlp_delta(const float* __restrict__ P, const float* __restrict__ norm,
                const float* __restrict__ Tt, int n, const float* __restrict__ H1,
                const float* __restrict__ H2, const float* __restrict__ Yn,
                float* __restrict__ D1, float* __restrict__ D2, float* __restrict__ D3,
                double* __restrict__ loss_s) {
    __shared__ float d3[FOUT], e3[FOUT], d2[FH];
    const int smp = blockIdx.x, u = threadIdx.x;
    if (smp >= n) return;
    const float inv_n = 1.0f / (float)n;
    if (u < FOUT) {
        float smax = norm[NORM_OS];
        for (int k = 1; k < FOUT; ++k) smax = fmaxf(smax, norm[NORM_OS + k]);
        const float r = norm[NORM_OS + u] / smax, w = r * r;
        const float e = Yn[(long long)smp * FOUT + u] - Tt[(long long)smp * FOUT + u] / norm[NORM_OS + u];
        e3[u] = w * e * e;
        d3[u] = w * e * inv_n;
        D3[(long long)smp * FOUT + u] = w * e * inv_n;
    }
    __syncthreads();
    if (u == 0) {
        double l = 0.0;
        for (int k = 0; k < FOUT; ++k) l += 0.5 * (double)e3[k];
        loss_s[smp] = l;
    }
    float a = 0.0f;
    for (int k = 0; k < FOUT; ++k) a = fmaf(P[OFF_W3 + u * FOUT + k], d3[k], a);
    const float h2 = H2[(long long)smp * FH + u];
    const float g2 = a * (1.0f - h2 * h2);
    d2[u] = g2;
    D2[(long long)smp * FH + u] = g2;
    __syncthreads();
    a = 0.0f;
    for (int v = 0; v < FH; ++v) a = fmaf(P[OFF_W2 + u * FH + v], d2[v], a);
    const float h1 = H1[(long long)smp * FH + u];
    D1[(long long)smp * FH + u] = a * (1.0f - h1 * h1);
}

// Parameter gradient, one thread per parameter: dW[i][o] = sum_s a_s[i] d_s[o],
// db[o] = sum_s d_s[o], samples summed in order (deterministic).
__global__ void __launch_bounds__(256)
    k_mlp_grad(const float* __restrict__ norm, const float* __restrict__ X, int n,
               const float* __restrict__ H1, const float* __restrict__ H2,
               const float* __restrict__ D1, const float* __restrict__ D2,
               const float* __restrict__ D3, float* __restrict__ G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NPARAM) return;
    float acc = 0.0f;
    if (t < OFF_B1) {
        const int i = t / FH, o = t % FH;
        const float mu = norm[NORM_MU + i], is = norm[NORM_IS + i];
        for (int s = 0; s < n; ++s)
            acc = fmaf((X[(long long)s * FIN + i] - mu) * is, D1[(long long)s * FH + o], acc);
    } else if (t < OFF_W2) {
        const int o = t - OFF_B1;
        for (int s = 0; s < n; ++s) acc += D1[(long long)s * FH + o];
    } else if (t < OFF_B2) {
        const int i = (t - OFF_W2) / FH, o = (t - OFF_W2) % FH;
        for (int s = 0; s < n; ++s) acc = fmaf(H1[(long long)s * FH + i], D2[(long long)s * FH + o], acc);
    } else if (t < OFF_W3) {
        const int o = t - OFF_B2;
        for (int s = 0; s < n; ++s) acc += D2[(long long)s * FH + o];
    } else if (t < OFF_B3) {
        const int i = (t - OFF_W3) / FOUT, o = (t - OFF_W3) % FOUT;
        for (int s = 0; s < n; ++s)
            acc = fmaf(H2[(long long)s * FH + i], D3[(long long)s * FOUT + o], acc);
    } else {
        const int o = t - OFF_B3;
        for (int s = 0; s < n; ++s) acc += D3[(long long)s * FOUT + o];
    }
    G[t] = acc;
}

// loss = sum of the per-sample terms / n, summed in order
__global__ void k_mlp_loss(const double* __restrict__ loss_s, int n, double* __restrict__ loss) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double l = 0.0;
    for (int s = 0; s < n; ++s) l += loss_s[s];
    *loss = l / n;
}

// Adam (Kingma & Ba 2015) with bias correction; step t >= 1.
__global__ void k_adam(float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                       const float* __restrict__ G, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NPARAM) return;
    const float g = G[t];
    const float m = b1 * M[t] + (1.0f - b1) * g;
    const float v = b2 * V[t] + (1.0f - b2) * g * g;
    M[t] = m;
    V[t] = v;
    P[t] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// Input mean and 1/std (FP64 sums in sample order; std < 1e-6 -> 1) and the
// output scale: the RMS of each target (samples in order; floored at 1e-12).
__global__ void k_fit_norm(const float* __restrict__ X, const float* __restrict__ Tt, int n,
                           float* __restrict__ norm) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < FIN) {
        double s1 = 0.0;
        for (int s = 0; s < n; ++s) s1 += X[(long long)s * FIN + t];
        const double mu = s1 / n;
        double s2 = 0.0;
        for (int s = 0; s < n; ++s) {
            const double d = X[(long long)s * FIN + t] - mu;
            s2 += d * d;
        }
        const double sd = sqrt(s2 / n);
        norm[NORM_MU + t] = (float)mu;
        norm[NORM_IS + t] = (float)(sd > 1e-6 ? 1.0 / sd : 1.0);
    } else if (t < FIN + FOUT) {
        const int k = t - FIN;
        double s2 = 0.0;
        for (int s = 0; s < n; ++s) {
            const double v = Tt[(long long)s * FOUT + k];
            s2 += v * v;
        }
        const double r = sqrt(s2 / n);
        norm[NORM_OS + k] = (float)(r > 1e-12 ? r : 1e-12);
    }
}

// F += dF * rho0 u_ref^2 D^2, T += dT * rho0 u_ref^2 D^3 (one thread per particle)
__global__ void k_apply_correction(const float* __restrict__ Y, const DevParticle* __restrict__ parts,
                                   int np, double u_ref, double rho0, double* __restrict__ force) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double D = parts[p].d, fs = rho0 * u_ref * u_ref * D * D, ts = fs * D;
    for (int a = 0; a < 3; ++a) {
        force[6 * p + a] += (double)Y[FOUT * p + a] * fs;
        force[6 * p + 3 + a] += (double)Y[FOUT * p + 3 + a] * ts;
    }
}

template <typename T>
cudaError_t features_t(const void* state, const Launch& L, const double* force, double u_ref,
                       float* feat) {
    const GeoMap gm{L.map, L.map_ext[0], L.map_ext[1], L.map_ext[2]};
    k_features<T><<<L.cp.np, 128, 0, L.stream>>>((const T*)state, L.g, L.cp, L.parts, gm, force,
                                                  u_ref, feat);
    return cudaGetLastError();
}

cudaError_t launch_features(int storage, const void* state, const Launch& L, const double* force,
                            double u_ref, float* feat) {
    if (L.cp.np < 1) return cudaSuccess;
    switch (storage) {
        case 1: return features_t<float>(state, L, force, u_ref, feat);
        case 4: return features_t<__half>(state, L, force, u_ref, feat);
        case 5: return features_t<__nv_bfloat16>(state, L, force, u_ref, feat);
        default: return features_t<double>(state, L, force, u_ref, feat);
    }
}

cudaError_t launch_apply_correction(const float* y, const DevParticle* parts, int np, double u_ref,
                                    double rho0, double* force, cudaStream_t s) {
    if (np < 1) return cudaSuccess;
    k_apply_correction<<<1, 32, 0, s>>>(y, parts, np, u_ref, rho0, force);
    return cudaGetLastError();
}

}  // namespace lbmgpu

// ---------------------------------------------------------------------------
// host side
struct lbm_mlp {
    cudaStream_t stream;
    float* params;  // NPARAM
    float* m;       // Adam first moment
    float* v;       // Adam second moment
    float* grad;    // NPARAM
    float* norm;    // NNORM
    double* loss;   // 1
    int adam_t;
    // per-sample work buffers (grown on demand)
    int cap;
    float *h1, *h2, *yn, *d1, *d2, *d3;
    double* loss_s;
    char err[512];
};

namespace {

lbm_status mfail(lbm_mlp* m, lbm_status st, const char* msg) {
    if (m) std::snprintf(m->err, sizeof(m->err), "%s", msg);
    return st;
}

lbm_status mcuda(lbm_mlp* m, cudaError_t e, const char* where) {
    if (m) std::snprintf(m->err, sizeof(m->err), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define MK(m, call, where)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return mcuda(m, e_, where);  \
    } while (0)

void free_work(lbm_mlp* m) {
    cudaFree(m->h1);
    cudaFree(m->h2);
    cudaFree(m->yn);
    cudaFree(m->d1);
    cudaFree(m->d2);
    cudaFree(m->d3);
    cudaFree(m->loss_s);
    m->h1 = m->h2 = m->yn = m->d1 = m->d2 = m->d3 = nullptr;
    m->loss_s = nullptr;
    m->cap = 0;
}

lbm_status ensure_work(lbm_mlp* m, int n) {
    if (n <= m->cap) return LBM_OK;
    MK(m, cudaStreamSynchronize(m->stream), "mlp sync");
    free_work(m);
    const size_t N = (size_t)n;
    MK(m, cudaMalloc(&m->h1, sizeof(float) * N * FH), "cudaMalloc mlp work");
    MK(m, cudaMalloc(&m->h2, sizeof(float) * N * FH), "cudaMalloc mlp work");
    MK(m, cudaMalloc(&m->yn, sizeof(float) * N * FOUT), "cudaMalloc mlp work");
    MK(m, cudaMalloc(&m->d1, sizeof(float) * N * FH), "cudaMalloc mlp work");
    MK(m, cudaMalloc(&m->d2, sizeof(float) * N * FH), "cudaMalloc mlp work");
    MK(m, cudaMalloc(&m->d3, sizeof(float) * N * FOUT), "cudaMalloc mlp work");
    MK(m, cudaMalloc(&m->loss_s, sizeof(double) * N), "cudaMalloc mlp work");
    m->cap = n;
    return LBM_OK;
}

// forward + deltas + parameter gradient into m->grad and the loss into m->loss
lbm_status gradient(lbm_mlp* m, const float* x, const float* t, int n) {
    lbm_status st = ensure_work(m, n);
    if (st != LBM_OK) return st;
    k_mlp_forward<<<n, FH, 0, m->stream>>>(m->params, m->norm, x, n, m->h1, m->h2, m->yn, nullptr,
                                           0.0f);
    MK(m, cudaGetLastError(), "mlp forward launch");
    k_mlp_delta<<<n, FH, 0, m->stream>>>(m->params, m->norm, t, n, m->h1, m->h2, m->yn, m->d1, m->d2,
                                         m->d3, m->loss_s);
    MK(m, cudaGetLastError(), "mlp delta launch");
    k_mlp_grad<<<(NPARAM + 255) / 256, 256, 0, m->stream>>>(m->norm, x, n, m->h1, m->h2, m->d1, m->d2,
                                                            m->d3, m->grad);
    MK(m, cudaGetLastError(), "mlp gradient launch");
    k_mlp_loss<<<1, 1, 0, m->stream>>>(m->loss_s, n, m->loss);
    MK(m, cudaGetLastError(), "mlp loss launch");
    return LBM_OK;
}

lbm_status read_loss(lbm_mlp* m, double* loss) {
    if (!loss) return LBM_OK;
    MK(m, cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream), "loss copy");
    MK(m, cudaStreamSynchronize(m->stream), "loss sync");
    return LBM_OK;
}

}  // namespace

namespace lbmgpu {
// used by the coupled step (lbm_api.cu): y = MLP(x) for n samples on stream s
cudaError_t mlp_infer(const lbm_mlp* m, const float* x, int n, float* y, float clip,
                      cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    k_mlp_forward<<<n, FH, 0, s>>>(m->params, m->norm, x, n, nullptr, nullptr, nullptr, y, clip);
    return cudaGetLastError();
}
}  // namespace lbmgpu

extern "C" {

lbm_status lbm_mlp_create(void* stream, lbm_mlp** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_mlp* m = new (std::nothrow) lbm_mlp();
    if (!m) return LBM_ERR_OOM;
    m->stream = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&m->params, sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = cudaMalloc(&m->norm, sizeof(float) * NNORM);
    if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(m->params, 0, sizeof(float) * NPARAM, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, sizeof(float) * NPARAM, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, sizeof(float) * NPARAM, m->stream);
    if (e == cudaSuccess) {
        // identity normalisation until set or fitted
        std::vector<float> nrm(NNORM, 1.0f);
        for (int i = 0; i < FIN; ++i) nrm[NORM_MU + i] = 0.0f;
        e = cudaMemcpy(m->norm, nrm.data(), sizeof(float) * NNORM, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        lbm_mlp_destroy(m);
        return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
    }
    *out = m;
    return LBM_OK;
}

void lbm_mlp_destroy(lbm_mlp* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    else cudaDeviceSynchronize();
    free_work(m);
    cudaFree(m->params);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->grad);
    cudaFree(m->norm);
    cudaFree(m->loss);
    delete m;
}

const char* lbm_mlp_last_error(const lbm_mlp* m) { return m ? m->err : "no model"; }

lbm_status lbm_mlp_set_params(lbm_mlp* m, const float* host, size_t count) {
    if (!m || !host) return LBM_ERR_ARG;
    if (count != (size_t)NPARAM) return mfail(m, LBM_ERR_ARG, "count must be LBM_MLP_PARAMS");
    MK(m, cudaMemcpyAsync(m->params, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, m->stream),
       "params upload");
    MK(m, cudaMemsetAsync(m->m, 0, sizeof(float) * NPARAM, m->stream), "adam reset");
    MK(m, cudaMemsetAsync(m->v, 0, sizeof(float) * NPARAM, m->stream), "adam reset");
    MK(m, cudaStreamSynchronize(m->stream), "params sync");
    m->adam_t = 0;
    return LBM_OK;
}

lbm_status lbm_mlp_get_params(lbm_mlp* m, float* host, size_t count) {
    if (!m || !host) return LBM_ERR_ARG;
    if (count != (size_t)NPARAM) return mfail(m, LBM_ERR_ARG, "count must be LBM_MLP_PARAMS");
    MK(m, cudaMemcpyAsync(host, m->params, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->stream),
       "params download");
    MK(m, cudaStreamSynchronize(m->stream), "params sync");
    return LBM_OK;
}

lbm_status lbm_mlp_set_normalization(lbm_mlp* m, const float* host, size_t count) {
    if (!m || !host) return LBM_ERR_ARG;
    if (count != (size_t)NNORM) return mfail(m, LBM_ERR_ARG, "count must be LBM_MLP_NORM");
    MK(m, cudaMemcpyAsync(m->norm, host, sizeof(float) * NNORM, cudaMemcpyHostToDevice, m->stream),
       "normalisation upload");
    MK(m, cudaStreamSynchronize(m->stream), "normalisation sync");
    return LBM_OK;
}

lbm_status lbm_mlp_get_normalization(lbm_mlp* m, float* host, size_t count) {
    if (!m || !host) return LBM_ERR_ARG;
    if (count != (size_t)NNORM) return mfail(m, LBM_ERR_ARG, "count must be LBM_MLP_NORM");
    MK(m, cudaMemcpyAsync(host, m->norm, sizeof(float) * NNORM, cudaMemcpyDeviceToHost, m->stream),
       "normalisation download");
    MK(m, cudaStreamSynchronize(m->stream), "normalisation sync");
    return LBM_OK;
}

lbm_status lbm_mlp_fit_normalization(lbm_mlp* m, const float* x_dev, const float* t_dev, int n) {
    if (!m || !x_dev || !t_dev || n < 1) return mfail(m, LBM_ERR_ARG, "need samples");
    k_fit_norm<<<(FIN + FOUT + 127) / 128, 128, 0, m->stream>>>(x_dev, t_dev, n, m->norm);
    MK(m, cudaGetLastError(), "normalisation launch");
    return LBM_OK;
}

lbm_status lbm_mlp_forward(lbm_mlp* m, const float* x_dev, int n, float* y_dev) {
    if (!m || !x_dev || !y_dev || n < 0) return mfail(m, LBM_ERR_ARG, "null buffer");
    MK(m, mlp_infer(m, x_dev, n, y_dev, 0.0f, m->stream), "mlp forward launch");
    return LBM_OK;
}

lbm_status lbm_mlp_gradient(lbm_mlp* m, const float* x_dev, const float* t_dev, int n,
                            float* grad_host, size_t count, double* loss) {
    if (!m || !x_dev || !t_dev || n < 1) return mfail(m, LBM_ERR_ARG, "need samples");
    if (grad_host && count != (size_t)NPARAM) return mfail(m, LBM_ERR_ARG, "count must be LBM_MLP_PARAMS");
    lbm_status st = gradient(m, x_dev, t_dev, n);
    if (st != LBM_OK) return st;
    if (grad_host) {
        MK(m, cudaMemcpyAsync(grad_host, m->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->stream),
           "gradient download");
        MK(m, cudaStreamSynchronize(m->stream), "gradient sync");
    }
    return read_loss(m, loss);
}

lbm_status lbm_mlp_train(lbm_mlp* m, const float* x_dev, const float* t_dev, int n, int steps,
                         float lr, double* loss) {
    if (!m || !x_dev || !t_dev || n < 1 || steps < 0 || !(lr > 0.0f))
        return mfail(m, LBM_ERR_ARG, "need samples, steps >= 0 and lr > 0");
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int it = 0; it < steps; ++it) {
        lbm_status st = gradient(m, x_dev, t_dev, n);
        if (st != LBM_OK) return st;
        ++m->adam_t;
        const float c1 = 1.0f - powf(b1, (float)m->adam_t), c2 = 1.0f - powf(b2, (float)m->adam_t);
        k_adam<<<(NPARAM + 255) / 256, 256, 0, m->stream>>>(m->params, m->m, m->v, m->grad, lr, b1, b2,
                                                           eps, c1, c2);
        MK(m, cudaGetLastError(), "adam launch");
    }
    return read_loss(m, loss);  // loss of the last step's parameters before its update
}

}  // extern "C"
