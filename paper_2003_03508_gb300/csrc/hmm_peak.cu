// Measured FP32 FFMA throughput of this GPU (the roofline denominator of the
// FP32-SIMT chunk kernel): every thread runs eight independent FFMA chains,
// so the FMA pipes, not latency, set the rate. Timed with CUDA events on a
// private stream; the chains' sums are stored so nothing is optimised away.
#include <cuda_runtime.h>

#include "hmm_internal.cuh"

namespace hmm {
namespace {

constexpr int PEAK_CHAINS = 8;

__global__ void __launch_bounds__(256) ffma_loop_kernel(int iters, float a, float b, float *out) {
    float x[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = (float)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace hmm

extern "C" int hmm_measure_fp32_peak(int device, double *tflops) {
    using namespace hmm;
    if (!tflops) return HMM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return HMM_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return HMM_ECUDA;
    const int threads = 256, blocks = sms * 8, iters = 4096;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HMM_ECUDA;
    if (cudaMalloc(&out, sizeof(float) * (size_t)threads * blocks) != cudaSuccess) return HMM_ENOMEM;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        float best = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 4 && ok; ++rep) {  // the first run is a warm-up
            cudaEventRecord(e0, st);
            ffma_loop_kernel<<<blocks, threads, 0, st>>>(iters, 0.999999f, 1e-7f, out);
            cudaEventRecord(e1, st);
            ok = cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess;
            float ms = 0.f;
            if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && rep > 0 && ms < best) best = ms;
        }
        if (ok && best < 1e30f) {
            const double flops = 2.0 * threads * (double)blocks * iters * 16 * PEAK_CHAINS;
            *tflops = flops / (best * 1e-3) / 1e12;
            rc = HMM_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    return rc;
}
