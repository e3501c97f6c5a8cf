// k_peaks.cu -- arithmetic rates of the current GPU, for stating which unit
// bounds a pass (no counterpart in the paper: a measurement utility).
//
// Each kernel runs eight independent FMA chains per thread (FP64 FMA, or FP32
// FMA) for a fixed number of iterations on 8 CTAs of 256 threads per SM; the
// chains' results are written out so nothing is optimised away.  Timed with
// CUDA events on the caller's stream after one untimed launch; the best of
// five launches is reported.  Clocks are whatever the GPU runs at.
#include "qf_host.h"

namespace qf {

constexpr int kRateIters = 4096;
constexpr int kRateChains = 8;

__global__ void __launch_bounds__(256) k_rate_f64(double *out, double a, double b) {
    double x[kRateChains];
#pragma unroll
    for (int i = 0; i < kRateChains; ++i) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < kRateIters; ++it)
#pragma unroll
        for (int i = 0; i < kRateChains; ++i) x[i] = fma(x[i], a, b);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kRateChains; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_rate_f32(float *out, float a, float b) {
    float x[kRateChains];
#pragma unroll
    for (int i = 0; i < kRateChains; ++i) x[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < kRateIters; ++it)
#pragma unroll
        for (int i = 0; i < kRateChains; ++i) x[i] = fmaf(x[i], a, b);
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kRateChains; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace qf

extern "C" qf_status qf_device_fma_rates(void *cuda_stream, double *fp64_fma_per_s, double *fp32_fma_per_s) {
    using namespace qf;
    if (!fp64_fma_per_s || !fp32_fma_per_s) return set_error(QF_ERR_ARG, "qf_device_fma_rates: output pointer is NULL");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int sms = device_sms();
    const int threads = 256, blocks = sms * 8;
    void *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)threads * blocks * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(QF_ERR_OOM, "qf_device_fma_rates: output buffer allocation failed");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    qf_status st = QF_OK;
    double best[2] = {0.0, 0.0};
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = set_error(QF_ERR_CUDA, "qf_device_fma_rates: event creation failed");
    } else {
        for (int kind = 0; kind < 2 && st == QF_OK; ++kind) {
            for (int r = 0; r < 6 && st == QF_OK; ++r) {
                cudaEventRecord(e0, stream);
                if (kind == 0) k_rate_f64<<<blocks, threads, 0, stream>>>((double *)buf, 0.999, 1e-3);
                else k_rate_f32<<<blocks, threads, 0, stream>>>((float *)buf, 0.999f, 1e-3f);
                cudaEventRecord(e1, stream);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaGetLastError();
                if (e != cudaSuccess) {
                    st = cuda_error(e, "qf_device_fma_rates");
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                const double rate = (double)threads * blocks * kRateIters * kRateChains / (ms * 1e-3);
                if (r > 0 && rate > best[kind]) best[kind] = rate;   // launch 0 warms up
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (st != QF_OK) return st;
    *fp64_fma_per_s = best[0];
    *fp32_fma_per_s = best[1];
    return QF_OK;
}
