// y = A_ff x together with the energy product x . y, for callers that must not
// allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is off limits -- inside a
// CUDA stream capture that another component owns, under an external memory
// manager that forbids allocations after start-up, or in a real-time loop
// where an allocation's latency or failure cannot be tolerated.  The fused
// SpMV-and-dot kernel reduces per-block partial sums through scratch memory;
// this entry point keeps that scratch in one file-scope device array instead
// of asking for memory, so it allocates nothing at all.
//
// The scratch array lives in every GPU that loads the library until the
// process exits (NOALLOC_MAX_BLOCKS * 8 bytes = 512 KiB).  All calls share it:
// two calls that overlap on the GPU (different streams, no ordering between
// them) race on it and give wrong dot products.  Every call writes all the
// partial sums it later reads, so nothing has to start at zero.
#include "ddg_internal.cuh"

#include <mutex>

namespace ddg {

constexpr int NOALLOC_T = 256;
constexpr int NOALLOC_MAX_BLOCKS = 65536;  // rows <= 65536 * 256 = 16,777,216

// file-scope scratch: one partial sum of x . (A x) per block
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS];

// device address of g_noalloc_partials on each device (host code may not use the symbol itself)
static double *g_partials_addr[64] = {nullptr};
static std::mutex g_partials_mu;

__global__ void __launch_bounds__(NOALLOC_T) k_spmv_dot_noalloc(const int *__restrict__ rowptr,
                                                                const int *__restrict__ col,
                                                                const double *__restrict__ val,
                                                                const double *__restrict__ x,
                                                                double *__restrict__ y, int n, double *partials) {
    __shared__ double sh[32];
    int i = blockIdx.x * NOALLOC_T + threadIdx.x;
    double v = 0.0;
    if (i < n) {
        double acc = 0.0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) acc += val[e] * x[col[e]];
        y[i] = acc;
        v = x[i] * acc;
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

__global__ void __launch_bounds__(NOALLOC_T) k_dot_final_noalloc(const double *partials, int nb, double *out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += NOALLOC_T) v += partials[b];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) *out = v;
}

// once per device, with that device current: look up the scratch array's device address
static int32_t partials_for_device(int device, double **out) {
    if (device < 0 || device >= 64) {
        set_error("device index out of range for the no-allocation scratch table");
        return DDG_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_partials_mu);
    if (!g_partials_addr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess || !ptr) {
            set_error(std::string("cudaGetSymbolAddress(no-allocation scratch): ") + cudaGetErrorString(e));
            return DDG_CUDA_ERROR;
        }
        g_partials_addr[device] = static_cast<double *>(ptr);
    }
    *out = g_partials_addr[device];
    return DDG_OK;
}

}  // namespace ddg

using namespace ddg;

extern "C" int32_t ddg_apply_A_dot_noalloc(ddg_problem *p, const double *x_dev, double *y_dev, double *xy_dev,
                                           ddg_stream stream) {
    return api_guard([&]() -> int32_t {
        clear_error();
        if (!p || !p->assembled || !x_dev || !y_dev || !xy_dev) {
            set_error("ddg_apply_A_dot_noalloc: NULL argument or problem not assembled");
            return DDG_INVALID_ARG;
        }
        const int nb = cdiv(p->nf, NOALLOC_T);
        if (nb > NOALLOC_MAX_BLOCKS) {
            set_error("ddg_apply_A_dot_noalloc: " + std::to_string(p->nf) + " rows exceed the limit of " +
                      std::to_string((long long)NOALLOC_MAX_BLOCKS * NOALLOC_T) + " rows");
            return DDG_TOO_LARGE;
        }
        DDG_CU(cudaSetDevice(p->ctx->device));
        double *partials = nullptr;
        DDG_TRY(partials_for_device(p->ctx->device, &partials));
        cudaStream_t s = stream ? (cudaStream_t)stream : p->stream;
        k_spmv_dot_noalloc<<<nb, NOALLOC_T, 0, s>>>(p->rowptr, p->col, p->val, x_dev, y_dev, p->nf, partials);
        DDG_LAUNCH_CHECK();
        k_dot_final_noalloc<<<1, NOALLOC_T, 0, s>>>(partials, nb, xy_dev);
        DDG_LAUNCH_CHECK();
        return DDG_OK;
    });
}
