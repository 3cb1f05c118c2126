// Measured FP64 arithmetic peak of the current GPU, the second roofline of
// the FP64 kernels (the refinement residual and the source term are bounded
// by min(HBM, FP64 throughput)).  Not part of the method: a measurement.
//
// Every thread runs kChains independent fused multiply-add chains
// (a = a * m + c) for `iters` steps, so the FP64 pipes stay busy without a
// dependency stall; the result is stored so nothing is optimised away.
#include <cuda_runtime.h>

#include <algorithm>

#include "fpconv.cuh"
#include "internal.cuh"

namespace {

constexpr int kChains = 8;
__device__ double g_probe_sink[1];

__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double m, double c) {
    double a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = (double)(threadIdx.x + q) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    if (s == 12345.678) g_probe_sink[0] = s;  // practically never true; keeps the chains live
}

// the integer-unit conversions of fpconv.cuh over caller-given inputs
__global__ void k_convert(const double* __restrict__ d_in, float* __restrict__ f_out, const float* __restrict__ f_in,
                          double* __restrict__ d_out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        f_out[i] = osm::f64_to_f32_rn(d_in[i]);
        d_out[i] = osm::f32_to_f64(f_in[i]);
    }
}

}  // namespace

extern "C" osmodi_status osmodi_probe_convert(const double* d_in, float* f_out, const float* f_in, double* d_out,
                                              int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!d_in || !f_out || !f_in || !d_out))) return OSMODI_E_INVALID;
    if (n == 0) return OSMODI_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    k_convert<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_in, f_out, f_in, d_out, n);
    OSM_CUDA(cudaGetLastError());
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_probe_fp64(double* gflops, double* ms, void* stream) {
    if (!gflops) return OSMODI_E_INVALID;
    int dev = 0, sms = 0, bps = 0;
    OSM_CUDA(cudaGetDevice(&dev));
    OSM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    OSM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_fp64_fma, 256, 0));
    const int grid = sms * (bps > 0 ? bps : 1);
    const int iters = 1 << 14;
    cudaStream_t s = (cudaStream_t)stream;
    // a damped map (|m| < 1) keeps the values finite
    k_fp64_fma<<<grid, 256, 0, s>>>(256, 0.999999, 1e-6);  // warm-up
    OSM_CUDA(cudaGetLastError());
    cudaEvent_t e0, e1;
    OSM_CUDA(cudaEventCreate(&e0));
    OSM_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, s);
        k_fp64_fma<<<grid, 256, 0, s>>>(iters, 0.999999, 1e-6);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            osm::set_cuda_error(e, "k_fp64_fma");
            return OSMODI_E_CUDA;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fmas = (double)grid * 256.0 * (double)iters * kChains;
    *gflops = 2.0 * fmas / (best * 1e-3) / 1e9;
    if (ms) *ms = best;
    return OSMODI_OK;
}
