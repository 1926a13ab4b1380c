// FMA throughput probe: the FP32 and FP64 fused multiply-add rates this GPU reaches, which the
// GNN kernel (FP32) and the Krylov kernels (FP64) are measured against.  No passage of the paper
// corresponds to it.
//
// Every thread runs CHAINS independent chains x <- x * a + b for ITERS steps (a slightly below 1,
// so the values stay normal), then stores the sum of its chains so that no chain is dead code.
// The grid holds 8 CTAs of 256 threads per SM: 64 warps per SM with 8 independent chains each
// cover the FMA latency many times over.  One warm-up launch, then one launch timed with CUDA
// events on the probe's own stream.
#include "ddg_internal.cuh"
#include "../../include/ddg_probe.h"

namespace ddg {

constexpr int PROBE_T = 256;
constexpr int PROBE_CTAS_PER_SM = 8;
constexpr int PROBE_CHAINS = 8;

__device__ __forceinline__ float fma_t(float x, float a, float b) { return fmaf(x, a, b); }
__device__ __forceinline__ double fma_t(double x, double a, double b) { return fma(x, a, b); }

template <class F, int ITERS>
__global__ void __launch_bounds__(PROBE_T) k_fma_probe(F a, F b, F *out) {
    F x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (F)(threadIdx.x + c) * (F)1e-3;
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma_t(x[c], a, b);
    }
    F s = 0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
    out[(size_t)blockIdx.x * PROBE_T + threadIdx.x] = s;
}

template <class F, int ITERS>
static int32_t probe_one(int blocks, cudaStream_t s, F *out, double *tflops) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DDG_CU(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        DDG_CU(err);
    }
    const F a = (F)0.999999, b = (F)1e-6;
    float ms = 0.f;
    k_fma_probe<F, ITERS><<<blocks, PROBE_T, 0, s>>>(a, b, out);  // warm-up
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    if (err == cudaSuccess) {
        k_fma_probe<F, ITERS><<<blocks, PROBE_T, 0, s>>>(a, b, out);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    DDG_CU(err);
    note_launches(2);
    const double flops = 2.0 * PROBE_CHAINS * (double)ITERS * (double)blocks * PROBE_T;
    *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return DDG_OK;
}

}  // namespace ddg

using namespace ddg;

extern "C" int32_t ddg_probe_fma_peaks(int32_t device, double *fp32_tflops, double *fp64_tflops) {
    return api_guard([&]() -> int32_t {
        clear_error();
        if (!fp32_tflops || !fp64_tflops) {
            set_error("ddg_probe_fma_peaks: NULL argument");
            return DDG_INVALID_ARG;
        }
        int count = 0;
        DDG_CU(cudaGetDeviceCount(&count));
        if (device < 0 || device >= count) {
            set_error("ddg_probe_fma_peaks: no such CUDA device");
            return DDG_INVALID_ARG;
        }
        DDG_CU(cudaSetDevice(device));
        int sms = 0;
        DDG_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        const int blocks = sms * PROBE_CTAS_PER_SM;
        cudaStream_t s = nullptr;
        DDG_CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        void *out = nullptr;
        cudaError_t err = cudaMalloc(&out, sizeof(double) * (size_t)blocks * PROBE_T);
        if (err != cudaSuccess) {
            cudaStreamDestroy(s);
            DDG_CU(err);
        }
        // FP32: 65,536 steps per chain, 0.32 TFLOP (about 5 ms at full rate; the compiler may pair
        // the chains into two-lane FMAs); FP64, at about 1/64 of that rate: 2,048 steps (about 9 ms)
        int32_t st = probe_one<float, 65536>(blocks, s, static_cast<float *>(out), fp32_tflops);
        if (st == DDG_OK) st = probe_one<double, 2048>(blocks, s, static_cast<double *>(out), fp64_tflops);
        cudaStreamSynchronize(s);
        cudaFree(out);
        cudaStreamDestroy(s);
        return st;
    });
}
