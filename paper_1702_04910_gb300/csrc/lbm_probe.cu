// Throughput probe of the FP64 pipe (declaration in include/lbm_gb300.h).
//
// The FP64 sweep of the library is bound by the rate at which the GPU issues
// FP64 instructions (GB300: a few FP64 lane-operations per SM per cycle,
// far below its FP32 rate), so its roofline needs that rate as measured on
// the device, not a nominal figure.  The probe runs independent chains of
// fused multiply-adds a <- a b + c in every thread of a grid that fills every
// SM, times the launch with CUDA events and returns DFMA lane-operations per
// second.  b < 1 and c > 0 keep every chain bounded (a -> c / (1 - b)).
#include <cuda_runtime.h>

#include "../../include/lbm_gb300.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__device__ double g_probe_sink;

__global__ void __launch_bounds__(PROBE_THREADS)
    k_dfma_rate(int iters, double b, double c, double never) {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = 1e-9 * threadIdx.x + i;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    if (s == never) g_probe_sink = s;  // never true: keeps every chain live
}

}  // namespace

extern "C" lbm_status lbm_measure_fp64_rate(void* stream, double* dfma_per_second) {
    if (!dfma_per_second) return LBM_ERR_ARG;
    *dfma_per_second = 0.0;
    int dev = 0, sms = 0, per_sm = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_rate, PROBE_THREADS, 0) !=
            cudaSuccess ||
        per_sm < 1)
        return LBM_ERR_CUDA;
    const int grid = sms * per_sm;
    const int iters = 2048;
    const double b = 1.0 - 1.0 / (1 << 20), c = 1.0 / (1 << 30);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return LBM_ERR_CUDA;
    }
    float best = 0.0f;
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // rep 0 warms up
        k_dfma_rate<<<grid, PROBE_THREADS, 0, s>>>(iters, b, c, -1.0);
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            k_dfma_rate<<<grid, PROBE_THREADS, 0, s>>>(iters, b, c, -1.0);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || !(best > 0.0f)) return LBM_ERR_CUDA;
    const double ops = (double)grid * PROBE_THREADS * PROBE_CHAINS * (double)iters;
    *dfma_per_second = ops / (best * 1e-3);
    return LBM_OK;
}
