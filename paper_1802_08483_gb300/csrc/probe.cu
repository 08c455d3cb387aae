// FP32 FMA throughput probe: the arithmetic roof the decoder's kernels are
// reported against.  Every thread runs kChains independent FMA recurrences
// (enough independent instructions to cover the FMA latency on every
// scheduler), the grid fills every SM several times over, and the host times
// the launch with CUDA events on its own stream.  Not part of the decoding
// method; the values stay bounded (|a| < 1) and are kept live by a
// data-dependent store that never fires in practice.
#include <cuda_runtime.h>

#include "../../include/mapdec.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_ffma_probe(float *out, int iters, float a,
                                                              float c) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-6f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0f) out[blockIdx.x] = s;  // never true: x stays positive
}

}  // namespace

extern "C" int mapdec_fp32_fma_peak(double *tflops_out, void *cuda_stream) {
    if (!tflops_out) return MAPDEC_ERR_ARG;
    *tflops_out = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MAPDEC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MAPDEC_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MAPDEC_ERR_CUDA;
    const int blocks = sms * 8;
    const int iters = 20000;
    if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess) return MAPDEC_ERR_NOMEM;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        k_ffma_probe<<<blocks, kProbeThreads, 0, st>>>(out, iters / 10, 0.9999f, 1e-7f);  // warm-up
        cudaEventRecord(e0, st);
        k_ffma_probe<<<blocks, kProbeThreads, 0, st>>>(out, iters, 0.9999f, 1e-7f);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
            const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * kProbeThreads;
            *tflops_out = flops / (ms * 1e-3) / 1e12;
            rc = MAPDEC_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}
